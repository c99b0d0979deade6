"""Adjoint of the SDC step (sdc_step_backward behind torch.autograd) against
finite differences, on the GPU forward and on the FP64 CPU oracle.

Three losses:
  * the released nuclear energy L = dV sum_zones (rhoE(t_f) - rhoE(t_0)) of the
    hot-spot box, differentiated with respect to the rate prefactors a_j and the
    initial temperature field;
  * the mass of each product species A_1 .. A_{n-1} at t_f (the yields), whose
    Jacobian with respect to a resolves every rate, also those that barely
    change the released energy;
  * a seeded random weighting L = sum w . (U(t_f) - U_b(t_f)) of the whole final
    state of a smooth, tie-free state, differentiated with respect to every
    initial field (U_b(t_f) is the unperturbed final state, subtracted so that
    the two runs of a difference cancel exactly outside the perturbation's
    domain of influence, and round-off stays near eps |U| / h).

The MC limiter is piecewise linear in the one-sided differences: at a tie
(dl = 0, dr = 0, or a switch between 2|dl|, 2|dr| and |dc|) the step has no
derivative, and the adjoint returns the derivative of the branch the primal
values select.  The hot-spot box is built on exact ties (a uniform background,
a mirror-symmetric spot), so its temperature gradients are compared with the
unlimited (centred-slope) scheme, which is smooth; its rate gradients, whose
perturbations leave the ties in place, are compared with both.  On the smooth
random state the MC-limited gradient is compared at sampled (field, zone)
entries whose finite differences at two step sizes agree (no branch switch
inside the step), with a floor on how many samples qualify.

Differences: fourth order, (8 (f(h) - f(-h)) - (f(2h) - f(-2h))) / 12h; with
relative steps 1e-4 (released energy) and 1e-6 (weighted state) both truncation
and round-off stay far below the 1e-6 tolerance.

The released energy is also taken in its binding-energy form,
L_b = dV sum_zones sum_i b_i (rho Y_i(t_f) - rho Y_i(t_0)) with
sum_i b_i s_ij = Q_j: total energy less the binding energy is conserved, so
L_b equals L, but it is a sum of the products' masses and does not cancel
(L is a difference of two sums of rho E, whose round-off, about eps sum |rho E|,
divided by the step of a difference, caps the plain central difference at h =
1e-6 near 1e-4).  With L_b the plain central difference at the relative step
h = 1e-6 agrees with the adjoint to 1e-6, for the rate prefactors and for the
initial temperature."""
import copy

import numpy as np
import pytest

import oracle as O
from paper_1910_12578_gb300 import workloads as W

pytestmark = pytest.mark.gpu

H = 1e-4        # relative step for the released-energy loss
H_STATE = 1e-6  # relative step for the weighted-state loss
H_PLAIN = 1e-6  # relative step of the plain central difference
TOL = 1e-6


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_12578_gb300 import build
    build.build()
    return torch


# ------------------------------------------------------------------ inputs
def hot_spot_problem(n, limiter, nodes="lobatto", nspec=7, n_iters=3):
    """nodes: "lobatto", "radau" (3 nodes) or "radau4" (node 0 and three Radau points)."""
    P, U = W.config_box(n=n, nspec=nspec, n_iters=n_iters, seed=1, T0=0.5)
    P = copy.deepcopy(P)
    P.limiter = limiter
    P.nodes = "radau" if nodes == "radau4" else nodes
    if nodes == "radau4":
        P.n_nodes = 4
    return P, U


def state_from_T(P, T):
    """Initial state of the hot-spot box with the given temperature field."""
    shp = T.shape
    rho = np.ones(shp)
    vel = [0.1 * np.ones(shp), np.zeros(shp), np.zeros(shp)]
    X = [np.ones(shp)] + [np.zeros(shp) for _ in range(P.net.nspec - 1)]
    return W.conserved_from(P.gamma, rho, vel, T, X)


def base_T(P):
    U = W.hot_spot_state(P, 2.0, T0=0.5)
    rho = U[0]
    ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho
    return (P.gamma - 1) * (U[4] - ke) / rho


def smooth_field(rng, shp):
    """Sum of three periodic plane waves with seeded wave vectors and phases,
    scaled to max |f| = 1."""
    n2, n1, n0 = shp
    z, y, x = np.meshgrid(np.arange(n2) / n2, np.arange(n1) / n1, np.arange(n0) / n0, indexing="ij")
    f = np.zeros(shp)
    for _ in range(3):
        k = rng.integers(-1, 2, 3)
        if not k.any():
            k[rng.integers(0, 3)] = 1
        f += rng.uniform(0.5, 1.0) * np.sin(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + rng.uniform(0, 2 * np.pi))
    return f / np.abs(f).max()


def generic_state(P, seed):
    """Smooth state without ties: the hot-spot temperature modulated by 10%,
    density 1 +- 0.1, a mean flow in every direction (no sonic or contact
    sign change at any face) with 0.03 modulation, and a smooth positive
    composition with X_0 between 0.7 and 0.9 (a field that is uniform up to
    rounding would leave the limiter's branch to rounding)."""
    rng = np.random.default_rng(seed)
    shp = (P.n[2], P.n[1], P.n[0])
    Th = base_T(P)
    rho = 1.0 + 0.1 * smooth_field(rng, shp)
    vel = [m + 0.03 * smooth_field(rng, shp) for m in (0.1, 0.08, 0.06)]
    T = Th * (1.0 + 0.1 * smooth_field(rng, shp))
    ns = P.net.nspec
    c = rng.uniform(0.5, 1.0, ns - 1)
    Xo = np.stack([c[i] * (1.0 + 0.5 * smooth_field(rng, shp)) for i in range(ns - 1)])
    Xo *= 0.2 * (1.0 + 0.5 * smooth_field(rng, shp)) / Xo.sum(0)   # X_0 varies too (0.7 .. 0.9)
    X = [1.0 - Xo.sum(0)] + list(Xo)
    return W.conserved_from(P.gamma, rho, vel, T, X)


def released(P, U0, U1):
    dV = P.dx[0] * P.dx[1] * P.dx[2]
    return dV * np.sum(U1[4] - U0[4])


def binding_weights(P):
    """dV b_i / mass_i per reactive species field: L_b = sum_i w_i sum_z rho X_i."""
    dV = P.dx[0] * P.dx[1] * P.dx[2]
    return dV * P.net.binding() / np.asarray(P.net.mass, dtype=np.float64)


def released_binding(P, U0, U1):
    """The released energy from the binding energies of the species made."""
    w = binding_weights(P)
    s = 2 + P.dim
    d = (U1[s:s + P.net.nspec] - U0[s:s + P.net.nspec]).reshape(P.net.nspec, -1).sum(1)
    return float(np.sum(w * d))


def fd(f, x, h):
    return (8.0 * (f(x + h) - f(x - h)) - (f(x + 2 * h) - f(x - 2 * h))) / (12.0 * h)


def fd_plain(f, x, h):
    return (f(x + h) - f(x - h)) / (2 * h)


# ------------------------------------------------------------------ models
class GpuModel:
    """Forward runs through sdc_step, gradients through sdc_step_fn (autograd)."""

    def __init__(self, torch, P, nsteps, dt):
        from paper_1910_12578_gb300 import sdc
        self.torch, self.sdc, self.P, self.nsteps, self.dt = torch, sdc, P, nsteps, dt
        self.ctx = sdc.Context(P)
        self._a = None

    def run(self, U0, a):
        torch = self.torch
        a = np.asarray(a, dtype=np.float64)
        if self._a is None or not np.array_equal(a, self._a):
            self.ctx.set_rates(a)
            self._a = a.copy()
        U = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
        for _ in range(self.nsteps):
            self.ctx.step(U, self.dt, stats=False)
        torch.cuda.synchronize()
        return U.cpu().numpy()

    def grad(self, U0, a, loss):
        """loss(U0_tensor, U_final_tensor) -> scalar tensor; returns (L, dL/dU0, dL/da)."""
        torch = self.torch
        Ut = torch.from_numpy(np.ascontiguousarray(U0)).cuda().requires_grad_(True)
        at = torch.tensor(np.asarray(a, dtype=np.float64), device="cuda", requires_grad=True)
        U = Ut
        for _ in range(self.nsteps):
            U = self.sdc.sdc_step_fn(U, at, self.ctx, self.dt)
        L = loss(Ut, U)
        L.backward()
        self._a = None  # sdc_step_fn sets the rates itself
        return float(L.item()), Ut.grad.cpu().numpy(), at.grad.cpu().numpy()


class OracleModel:
    def __init__(self, P, nsteps, dt):
        self.P, self.nsteps, self.dt = copy.deepcopy(P), nsteps, dt

    def run(self, U0, a):
        self.P.net.a = np.asarray(a, dtype=np.float64)
        o = O.Oracle(self.P)
        V = np.array(U0, copy=True)
        for _ in range(self.nsteps):
            V, _ = o.step(V, self.dt)
        return V


def released_loss(P):
    dV = P.dx[0] * P.dx[1] * P.dx[2]
    return lambda U0, U: dV * (U[4] - U0[4]).sum()


def binding_loss(P):
    w = binding_weights(P)
    s = 2 + P.dim

    def f(U0, U):
        import torch
        wt = torch.tensor(w, dtype=torch.float64, device=U.device)
        d = (U[s:s + P.net.nspec] - U0[s:s + P.net.nspec]).reshape(P.net.nspec, -1).sum(1)
        return (wt * d).sum()
    return f


def T_gradient(P, U0, gU0):
    """dL/dT from dL/dU0 (the temperature enters rhoE = rho T / (gamma - 1) + kinetic)."""
    return gU0[4] * U0[0] / (P.gamma - 1)


# ------------------------------------------------------------------ tests
def vjp_case(name, limiter):
    if name == "1d":
        P, U = W.config_1d()
    elif name == "box16":
        P, U = W.config_box(n=16, nspec=7, n_iters=3, seed=1, T0=0.5)
    else:
        P, _ = W.config_box(n=16, nspec=7, n_iters=3, seed=1, T0=0.5)
        U = None
    P = copy.deepcopy(P)
    P.limiter = limiter
    if U is None:
        U = generic_state(P, 5)
    return P, U


@pytest.mark.parametrize("name,limiter", [("1d", 1), ("box16", 0), ("smooth16", 0), ("smooth16", 1)])
def test_advective_vjp_reverse_sweep_matches_forward_mode(torch_cuda, name, limiter):
    """sdc_advective_term_vjp: the reverse sweep per face (mode 0, used by the
    backward step) against forward-mode dual numbers (mode 1), and accumulation.
    The two round u = m / rho and p differently, so a limiter tie that only
    rounding separates may take different branches in the two: the MC cases
    use states whose neighbouring values differ far above rounding (the
    hot-spot box's far field does not)."""
    torch = torch_cuda
    from paper_1910_12578_gb300 import sdc
    P, U = vjp_case(name, limiter)
    ctx = sdc.Context(P)
    Ud = torch.from_numpy(U).cuda()
    Ab = torch.from_numpy(np.random.default_rng(4).normal(size=U.shape)).cuda()
    g0, g1 = torch.zeros_like(Ud), torch.zeros_like(Ud)
    ctx.advective_term_vjp(Ud, Ab, g0, 0)
    ctx.advective_term_vjp(Ud, Ab, g1, 1)
    torch.cuda.synchronize()
    a, b = g0.cpu().numpy(), g1.cpu().numpy()
    scale = np.abs(b).reshape(b.shape[0], -1).max(1)
    err = (np.abs(a - b).reshape(b.shape[0], -1).max(1) / np.maximum(scale, 1e-300 + 1e-12 * scale.max())).max()
    print(name, "limiter", limiter, "reverse vs forward mode:", err)
    assert np.isfinite(a).all()
    assert err <= 1e-12
    ctx.advective_term_vjp(Ud, Ab, g0, 0)
    torch.cuda.synchronize()
    assert np.array_equal(g0.cpu().numpy(), 2.0 * a)


def test_advective_vjp_matches_oracle_differences(torch_cuda):
    """v . (dA/dU)^T Abar against the fourth-order difference of Abar . A(U + t v)
    of the oracle's advective term (centred slopes).  The Davis wave speeds
    (min and max of the two sides' u -/+ c) switch sides on surfaces that cut
    many faces of a smooth 3D flow, so the difference uses a step of 1e-8
    relative, small enough to cross none of those switches (1e-6 crosses some:
    the differences then move by ~2e-6), with round-off near 3e-9."""
    torch = torch_cuda
    from paper_1910_12578_gb300 import sdc
    P, U = vjp_case("smooth16", 0)
    o = O.Oracle(P)
    rng = np.random.default_rng(8)
    Abar = rng.normal(size=U.shape)
    v = U * rng.normal(size=U.shape)
    ctx = sdc.Context(P)
    g = torch.zeros(U.shape, dtype=torch.float64, device="cuda")
    ctx.advective_term_vjp(torch.from_numpy(U).cuda(), torch.from_numpy(Abar).cuda(), g, 0)
    torch.cuda.synchronize()
    lhs = float(np.sum(v * g.cpu().numpy()))
    d = fd(lambda t: float(np.sum(Abar * o.advective(U + t * v))), 0.0, 1e-8)
    print("advective VJP vs oracle difference:", abs(lhs - d) / abs(d))
    assert abs(lhs - d) <= 1e-7 * abs(d)


def yields(P, U):
    """Mass of every product species A_1 .. A_{n-1} in the box."""
    dV = P.dx[0] * P.dx[1] * P.dx[2]
    return dV * U[2 + P.dim + 1:].reshape(P.net.nspec - 1, -1).sum(1)


def yield_loss(P, j):
    dV = P.dx[0] * P.dx[1] * P.dx[2]
    return lambda U0, U: dV * U[2 + P.dim + 1 + j].sum()


def rate_gradients(model, P, U0, a):
    """Adjoint dL/da for the released energy and the Jacobian of the product
    yields with respect to a (one backward pass per yield)."""
    L, _, ga = model.grad(U0, a, released_loss(P))
    J = np.stack([model.grad(U0, a, yield_loss(P, j))[2] for j in range(len(a))])
    return L, ga, J


def rate_differences(run, P, U0, a):
    d_rel, d_yield = [], []
    for k in range(len(a)):
        e = np.zeros_like(a); e[k] = 1.0
        d_rel.append(fd(lambda s: released(P, U0, run(U0, a + s * e)), 0.0, H * a[k]))
        d_yield.append(fd(lambda s: yields(P, run(U0, a + s * e)), 0.0, H * a[k]))
    return np.array(d_rel), np.stack(d_yield, axis=1)


def rate_errors(ga, d_rel, J, d_yield):
    """Released energy: max-norm error relative to the largest component (the
    weak reactions barely change the released energy, and their differences
    sit at its round-off).  Yields: every entry relative to itself, with a
    floor of 1e-2 of its row's largest entry (each rate is checked in full on
    the rows of the species it feeds).  Below that floor an entry sits at the
    differences' noise: every forward run rounds each zone's Newton iterate
    at about eps |w|, so a yield Y carries about eps |Y| of noise, and its
    difference quotient about eps |Y| / h, a few 1e-15 on the 32^3 box, where
    the smallest resolved entries (a weakly coupled rate on an early product)
    are ~1e-11 against row maxima ~1e-5."""
    err_rel = np.abs(ga - d_rel).max() / np.abs(d_rel).max()
    rowmax = np.abs(d_yield).max(axis=1, keepdims=True)
    err_y = np.abs(J - d_yield) / np.maximum(np.abs(d_yield), 1e-2 * rowmax)
    return err_rel, err_y


@pytest.mark.parametrize("n,nsteps,limiter,nodes", [(8, 2, 1, "lobatto"), (32, 5, 1, "lobatto"), (8, 2, 0, "lobatto"),
                                                    (32, 5, 0, "lobatto"), (8, 2, 1, "radau"), (8, 2, 1, "radau4")])
def test_rate_gradient_hot_spot(torch_cuda, n, nsteps, limiter, nodes):
    """dL/da_j of the released energy and of the product yields against GPU
    finite differences (Gauss-Lobatto and Radau node sets)."""
    P, U = hot_spot_problem(n, limiter, nodes)
    dt = O.Oracle(P).cfl_dt(U)
    model = GpuModel(torch_cuda, P, nsteps, dt)
    U0 = state_from_T(P, base_T(P))
    a = np.array(P.net.a, dtype=np.float64)
    L, ga, J = rate_gradients(model, P, U0, a)
    assert L == pytest.approx(released(P, U0, model.run(U0, a)), rel=1e-12)
    d_rel, d_yield = rate_differences(model.run, P, U0, a)
    err_rel, err_y = rate_errors(ga, d_rel, J, d_yield)
    # the binding-energy form: the same quantity, and the plain central
    # difference at h = 1e-6 for every prefactor
    Lb, _, gb = model.grad(U0, a, binding_loss(P))
    d_plain = []
    for k in range(len(a)):
        e = np.zeros_like(a); e[k] = 1.0
        d_plain.append(fd_plain(lambda s: released_binding(P, U0, model.run(U0, a + s * e)), 0.0, H_PLAIN * a[k]))
    d_plain = np.array(d_plain)
    err_plain = np.abs(gb - d_plain).max() / np.abs(d_plain).max()
    print("rate gradients vs FD: released", err_rel, "yields (max per row)", err_y.max(axis=1),
          "binding form, plain h=1e-6:", err_plain, "binding vs rho E form", np.abs(gb - ga).max() / np.abs(ga).max())
    assert np.isfinite(ga).all() and np.isfinite(J).all()
    assert err_rel <= TOL
    assert err_y.max() <= TOL
    assert Lb == pytest.approx(L, rel=1e-9)
    assert np.abs(gb - ga).max() <= TOL * np.abs(ga).max()
    assert err_plain <= TOL


@pytest.mark.parametrize("limiter", [1, 0])
def test_rate_gradient_13species(torch_cuda, limiter):
    """The 13-species chain (14 x 14 Newton system; the adjoint's transposed
    solve by the bordered chain elimination in reversed chain order): dL/da_j
    of the released energy and of the product yields against GPU finite
    differences and against the oracle's, 8^3, two steps of the 3-node, 4-iteration
    scheme; the binding-energy form against the plain central difference at
    h = 1e-6."""
    P, U = hot_spot_problem(8, limiter, nspec=13, n_iters=4)
    dt = O.Oracle(P).cfl_dt(U)
    model = GpuModel(torch_cuda, P, 2, dt)
    orc = OracleModel(P, 2, dt)
    U0 = state_from_T(P, base_T(P))
    a = np.array(P.net.a, dtype=np.float64)
    L, ga, J = rate_gradients(model, P, U0, a)
    assert L == pytest.approx(released(P, U0, model.run(U0, a)), rel=1e-12)
    d_rel, d_yield = rate_differences(model.run, P, U0, a)
    err_rel, err_y = rate_errors(ga, d_rel, J, d_yield)
    o_rel, o_yield = rate_differences(orc.run, P, U0, a)
    oerr_rel, oerr_y = rate_errors(ga, o_rel, J, o_yield)
    Lb, _, gb = model.grad(U0, a, binding_loss(P))
    d_plain = []
    for k in range(len(a)):
        e = np.zeros_like(a); e[k] = 1.0
        d_plain.append(fd_plain(lambda s: released_binding(P, U0, model.run(U0, a + s * e)), 0.0, H_PLAIN * a[k]))
    d_plain = np.array(d_plain)
    err_plain = np.abs(gb - d_plain).max() / np.abs(d_plain).max()
    print("13 species: released", err_rel, "yields", err_y.max(), "oracle FD: released", oerr_rel, "yields",
          oerr_y.max(), "binding plain h=1e-6", err_plain)
    assert np.isfinite(ga).all() and np.isfinite(J).all()
    assert err_rel <= TOL and err_y.max() <= TOL
    assert oerr_rel <= TOL and oerr_y.max() <= TOL
    assert Lb == pytest.approx(L, rel=1e-9)
    assert err_plain <= TOL


@pytest.mark.parametrize("n,nsteps", [(8, 2), (32, 5)])
def test_temperature_gradient_hot_spot_unlimited(torch_cuda, n, nsteps):
    """dL/dT of the released energy (centred slopes) at sampled zones, the
    spot's centre, and along a seeded random direction."""
    P, U = hot_spot_problem(n, 0)
    dt = O.Oracle(P).cfl_dt(U)
    model = GpuModel(torch_cuda, P, nsteps, dt)
    T = base_T(P)
    a = np.array(P.net.a, dtype=np.float64)
    U0 = state_from_T(P, T)
    _, gU0, _ = model.grad(U0, a, released_loss(P))
    gT = T_gradient(P, U0, gU0)
    loss = lambda Tx: released(P, state_from_T(P, Tx), model.run(state_from_T(P, Tx), a))
    rng = np.random.default_rng(0)
    zones = [tuple(rng.integers(0, n, 3)) for _ in range(6)] + [(n // 2, n // 2, n // 2)]
    scale = np.abs(gT).max()
    err = []
    for z in zones:
        e = np.zeros_like(T); e[z] = 1.0
        err.append(abs(gT[z] - fd(lambda s: loss(T + s * e), 0.0, H * T[z])) / scale)
    v = rng.choice([-1.0, 1.0], size=T.shape) * T
    d = fd(lambda s: loss(T + s * v), 0.0, H)
    err_dir = abs(float(np.sum(gT * v)) - d) / abs(d)
    # the binding-energy form with the plain central difference at h = 1e-6
    _, gUb, _ = model.grad(U0, a, binding_loss(P))
    gTb = T_gradient(P, U0, gUb)
    loss_b = lambda Tx: released_binding(P, state_from_T(P, Tx), model.run(state_from_T(P, Tx), a))
    scale_b = np.abs(gTb).max()
    err_b = []
    for z in zones:
        e = np.zeros_like(T); e[z] = 1.0
        err_b.append(abs(gTb[z] - fd_plain(lambda s: loss_b(T + s * e), 0.0, H_PLAIN * T[z])) / scale_b)
    d_b = fd_plain(lambda s: loss_b(T + s * v), 0.0, H_PLAIN)
    err_dir_b = abs(float(np.sum(gTb * v)) - d_b) / abs(d_b)
    print("temperature gradient vs FD:", err, "direction", err_dir, "binding form, plain h=1e-6:", err_b, err_dir_b)
    assert max(err) <= TOL
    assert err_dir <= TOL
    assert max(err_b) <= TOL
    assert err_dir_b <= TOL


def _sampled_state_gradient(model, P, U0, a, g, nsamples, seed):
    """(field, zone) samples of dL/dU0 for L = sum w (U(t_f) - U_b(t_f)) against
    differences at relative steps 10 H_STATE and H_STATE; returns the list of
    (gradient, difference, consistent)."""
    w = np.random.default_rng(seed).normal(size=U0.shape)
    Vb = model.run(U0, a)
    loss = lambda Ux: float(np.sum(w * (model.run(Ux, a) - Vb)))
    rng = np.random.default_rng(seed + 1)
    out = []
    for _ in range(nsamples):
        f = int(rng.integers(0, U0.shape[0]))
        z = tuple(int(i) for i in rng.integers(0, P.n[0], 3))
        e = np.zeros_like(U0); e[(f,) + z] = 1.0
        s = abs(U0[(f,) + z])
        d1 = fd(lambda t: loss(U0 + t * e), 0.0, 10 * H_STATE * s)
        d2 = fd(lambda t: loss(U0 + t * e), 0.0, H_STATE * s)
        consistent = abs(d1 - d2) <= 1e-7 * max(abs(d2), 1.0)
        out.append((g[(f,) + z], d2, consistent))
    return out, loss


@pytest.mark.parametrize("limiter", [0, 1])
def test_state_gradient_smooth_state(torch_cuda, limiter):
    """dL/dU0 of the weighted final state on a smooth 16^3 state, 2 steps:
    sampled entries against GPU differences (entries whose differences are
    self-consistent), and along a random direction for centred slopes."""
    torch = torch_cuda
    P, _ = hot_spot_problem(16, limiter)
    U0 = generic_state(P, 5)
    dt = O.Oracle(P).cfl_dt(U0)
    model = GpuModel(torch, P, 2, dt)
    a = np.array(P.net.a, dtype=np.float64)
    w = torch.from_numpy(np.random.default_rng(17).normal(size=U0.shape)).cuda()
    _, g, _ = model.grad(U0, a, lambda U0t, U: (w * U).sum())
    samples, loss = _sampled_state_gradient(model, P, U0, a, g, 32, 17)
    good = [(gi, d) for gi, d, c in samples if c]
    err = [abs(gi - d) / max(abs(d), 1e-2) for gi, d in good]
    print("limiter", limiter, "consistent samples", len(good), "of", len(samples), "max err", max(err))
    assert np.isfinite(g).all()
    assert len(good) >= (24 if limiter == 0 else 10)
    assert max(err) <= TOL
    if limiter == 0:
        v = U0 * np.random.default_rng(3).normal(size=U0.shape)
        d = fd(lambda t: loss(U0 + t * v), 0.0, 1e-7)
        assert abs(float(np.sum(g * v)) - d) <= TOL * abs(d)


def test_gradient_matches_oracle_finite_differences_8cubed(torch_cuda):
    """The GPU adjoint against differences of the FP64 CPU oracle on 8^3:
    rate prefactors and zone temperatures of the hot spot (centred slopes,
    5 steps), and sampled state entries of the smooth state (MC limiter,
    2 steps, self-consistent samples)."""
    torch = torch_cuda
    P, U = hot_spot_problem(8, 0)
    dt = O.Oracle(P).cfl_dt(U)
    nsteps = 5
    gpu, orc = GpuModel(torch, P, nsteps, dt), OracleModel(P, nsteps, dt)
    T = base_T(P)
    a = np.array(P.net.a, dtype=np.float64)
    U0 = state_from_T(P, T)
    _, gU0, _ = gpu.grad(U0, a, released_loss(P))
    gT = T_gradient(P, U0, gU0)
    _, ga, J = rate_gradients(gpu, P, U0, a)
    d_rel, d_yield = rate_differences(orc.run, P, U0, a)
    err_rel, err_y = rate_errors(ga, d_rel, J, d_yield)
    loss_T = lambda Tx: released(P, state_from_T(P, Tx), orc.run(state_from_T(P, Tx), a))
    scale = np.abs(gT).max()
    err_T = []
    for z in [(4, 4, 4), (3, 4, 5), (0, 0, 0), (4, 2, 6)]:
        e = np.zeros_like(T); e[z] = 1.0
        err_T.append(abs(gT[z] - fd(lambda s: loss_T(T + s * e), 0.0, H * T[z])) / scale)
    # smooth state, MC limiter
    Pm, _ = hot_spot_problem(8, 1)
    Um = generic_state(Pm, 5)
    dtm = O.Oracle(Pm).cfl_dt(Um)
    gm, om = GpuModel(torch, Pm, 2, dtm), OracleModel(Pm, 2, dtm)
    w = torch.from_numpy(np.random.default_rng(23).normal(size=Um.shape)).cuda()
    _, g, _ = gm.grad(Um, a, lambda U0t, Uf: (w * Uf).sum())
    samples, _ = _sampled_state_gradient(om, Pm, Um, a, g, 24, 23)
    good = [(gi, d) for gi, d, c in samples if c]
    err_s = [abs(gi - d) / max(abs(d), 1e-2) for gi, d in good]
    print("adjoint vs oracle FD: released", err_rel, "yields", err_y.max(axis=1), "T", err_T, "state", len(good),
          "of", len(samples), max(err_s))
    assert err_rel <= TOL
    assert err_y.max() <= TOL
    assert max(err_T) <= TOL
    assert len(good) >= 8
    assert max(err_s) <= TOL
