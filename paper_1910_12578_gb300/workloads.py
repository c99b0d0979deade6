"""Seeded synthetic workloads for the SDC hydro + reaction sweep.

This module only builds inputs: box geometry, the toy reaction networks and
their seeded constants, and the initial conserved state.  It holds none of the
method's arithmetic (no fluxes, rates, quadrature or Newton solve), so both the
CUDA path and the CPU oracle can consume its arrays.

The paper's own workloads (X-ray burst flames with a 13-isotope network and a
realistic EOS, section 4) need rate tables and EOS data that are not part of
the paper; these synthetic problems stand in for them with the same structure:
a stiff alpha-chain network heated by a hot spot inside a periodic box, or a
batch of ragged boxes.

Conserved field order: [rho, rho*u_0..rho*u_{dim-1}, rho*E, rho*X_0..].
Arrays are field-major, x fastest (numpy shape (nvar, n2, n1, n0)).
The initial state is set from (rho, u, T, X) with the gamma-law relation
p = rho*T, rho*E = p/(gamma-1) + rho|u|^2/2 that defines the workload.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

RATE_POWER = 0       # f_j(T) = T^nu_j
RATE_ARRHENIUS = 1   # f_j(T) = exp(-nu_j / T)


@dataclasses.dataclass
class Network:
    nspec: int
    rate_law: int
    mass: np.ndarray            # (nspec,) species mass numbers
    a: np.ndarray               # (nreac,) rate prefactors
    nu: np.ndarray              # (nreac,) temperature exponents / activation
    Q: np.ndarray               # (nreac,) energy released per unit rate
    reac: np.ndarray            # (nreac, 2) reactant species, -1 = none
    cnt: np.ndarray             # (nreac, 2) reactant multiplicities
    prod: np.ndarray            # (nreac,) product species

    @property
    def nreac(self) -> int:
        return int(self.a.shape[0])

    def binding(self) -> np.ndarray:
        """b_i with sum_i b_i s_ij = Q_j (b of the first species is 0).

        Only used to state the conserved total energy of a test; solved from
        the reaction list by forward substitution along the chain."""
        b = np.zeros(self.nspec)
        known = np.zeros(self.nspec, dtype=bool)
        known[0] = True
        for _ in range(self.nspec):
            for j in range(self.nreac):
                p = int(self.prod[j])
                if known[p]:
                    continue
                rs = [int(s) for s in self.reac[j] if s >= 0]
                if all(known[s] for s in rs):
                    b[p] = self.Q[j] + sum(b[int(self.reac[j][k])] * self.cnt[j][k]
                                           for k in range(2) if self.reac[j][k] >= 0)
                    known[p] = True
        return b


def decay_network(k0: float = 1e3, activation: float = 10.0, Q: float = 1.0) -> Network:
    """Single reaction A -> B with k(T) = k0 exp(-activation/T) and energy Q."""
    return Network(
        nspec=2, rate_law=RATE_ARRHENIUS,
        mass=np.array([1.0, 1.0]),
        a=np.array([k0]), nu=np.array([activation]), Q=np.array([Q]),
        reac=np.array([[0, -1]], dtype=np.int32), cnt=np.array([[1, 0]], dtype=np.int32),
        prod=np.array([1], dtype=np.int32))


def alpha_chain(nspec: int, rng: np.random.Generator) -> Network:
    """Toy alpha chain A0..A_{nspec-1}: 3 A0 -> A1, then A_i + A0 -> A_{i+1}.

    Masses [1, 3, 4, 5, ...] make every reaction conserve mass.  For each
    reaction in order the seed draws log10 a ~ U[-2, 2], nu ~ U[5, 20],
    Q ~ U[0.5, 5]."""
    nreac = nspec - 1
    mass = np.array([1.0] + [3.0 + i for i in range(nspec - 1)])
    a = np.empty(nreac); nu = np.empty(nreac); Q = np.empty(nreac)
    for j in range(nreac):
        a[j] = 10.0 ** rng.uniform(-2.0, 2.0)
        nu[j] = rng.uniform(5.0, 20.0)
        Q[j] = rng.uniform(0.5, 5.0)
    reac = np.full((nreac, 2), -1, dtype=np.int32)
    cnt = np.zeros((nreac, 2), dtype=np.int32)
    prod = np.zeros(nreac, dtype=np.int32)
    reac[0] = [0, -1]; cnt[0] = [3, 0]; prod[0] = 1
    for i in range(1, nreac):
        reac[i] = [i, 0]; cnt[i] = [1, 1]; prod[i] = i + 1
    return Network(nspec, RATE_POWER, mass, a, nu, Q, reac, cnt, prod)


@dataclasses.dataclass
class Problem:
    """One periodic box plus the network and the SDC parameters."""
    dim: int
    n: tuple                     # zones per axis (n0, n1, n2)
    dx: tuple
    gamma: float
    net: Network
    n_nodes: int = 3             # M (Gauss-Lobatto nodes)
    n_iters: int = 3             # K (SDC iterations)
    nodes: str = "lobatto"       # "lobatto" (Gauss-Lobatto) or "radau" (node 0 + Radau IIA points)
    space_order: int = 2         # 2: PLM/HLLC; 4: the fourth-order finite-volume operators
    limiter: int = 1             # 1 = MC, 0 = unlimited centred slopes
    newton_rtol: float = 1e-10
    newton_maxit: int = 100
    cfl: float = 0.5

    @property
    def nvar(self) -> int:
        return 2 + self.dim + self.net.nspec

    @property
    def nzones(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])


def conserved_from(gamma: float, rho, vel: List[np.ndarray], T, X: List[np.ndarray]) -> np.ndarray:
    """Initial conserved state from rho, velocity components, T and X."""
    p = rho * T
    ke = sum(0.5 * rho * v * v for v in vel)
    fields = [rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + ke] + [rho * x for x in X]
    return np.stack([np.ascontiguousarray(f, dtype=np.float64) for f in fields])


def _centres(n, dx):
    return (np.arange(n) + 0.5) * dx


def config_1d(nx: int = 64, seed: int = 0) -> tuple:
    """1D, 64 zones on [0,1], periodic, gamma = 5/3, rho = 1, u = 0.1,
    T = 1 + 0.2 exp(-(x-0.5)^2/0.01), X_A = 1, A -> B with k = 1e3 exp(-10/T),
    Q = 1; 2 nodes, 2 iterations, CFL 0.5."""
    net = decay_network()
    P = Problem(dim=1, n=(nx, 1, 1), dx=(1.0 / nx, 1.0, 1.0), gamma=5.0 / 3.0, net=net,
                n_nodes=2, n_iters=2)
    x = _centres(nx, 1.0 / nx)
    rho = np.ones(nx)
    T = 1.0 + 0.2 * np.exp(-(x - 0.5) ** 2 / 0.01)
    U = conserved_from(P.gamma, rho, [0.1 * np.ones(nx)], T, [np.ones(nx), np.zeros(nx)])
    return P, U.reshape(P.nvar, 1, 1, nx)


def hot_spot_state(P: Problem, amp: float, u0: float = 0.1, T0: float = 1.0) -> np.ndarray:
    """3D box [0, n*dx]^3: rho = 1, u = (u0, 0, 0), X_0 = 1, T = T0 (1 + (amp-1)
    exp(-|x - x_c|^2 / 0.01)) in coordinates scaled by the box length.  The
    offsets from the centre, (i + 1/2 - n/2) / n, are exact negatives of each
    other across the box's mid-planes, so the state is mirror-symmetric to the
    last bit (with n a power of two these are the centres less 1/2 exactly)."""
    n0, n1, n2 = P.n
    x, y, z = ((np.arange(m) + 0.5 - 0.5 * m) / m for m in (n0, n1, n2))
    Z, Y, Xc = np.meshgrid(z, y, x, indexing="ij")
    r2 = Xc ** 2 + Y ** 2 + Z ** 2
    T = T0 * (1.0 + (amp - 1.0) * np.exp(-r2 / 0.01))
    rho = np.ones_like(T)
    vel = [u0 * np.ones_like(T), np.zeros_like(T), np.zeros_like(T)]
    X = [np.ones_like(T)] + [np.zeros_like(T) for _ in range(P.net.nspec - 1)]
    return conserved_from(P.gamma, rho, vel, T, X)


def config_box(n: int = 64, nspec: int = 7, n_nodes: int = 3, n_iters: int = 3,
               amp: float = 2.0, seed: int = 0, dx: Optional[float] = None, T0: float = 1.0) -> tuple:
    """Single periodic n^3 box on the unit cube with the seeded alpha chain and
    a Gaussian hot spot (peak temperature amp x the background)."""
    rng = np.random.default_rng(seed)
    net = alpha_chain(nspec, rng)
    h = 1.0 / n if dx is None else dx
    P = Problem(dim=3, n=(n, n, n), dx=(h, h, h), gamma=5.0 / 3.0, net=net,
                n_nodes=n_nodes, n_iters=n_iters)
    return P, hot_spot_state(P, amp, T0=T0)


def shock_tube_state(P: Problem, axis: int, left, right, x0: float = 0.5) -> np.ndarray:
    """Planar Riemann problem along `axis`: (rho, u_axis, p) = `left` where the
    scaled coordinate x_axis / L is below x0, `right` above it; the other
    velocity components are zero and X_0 = 1.  The box is periodic, so a
    second, mirrored discontinuity sits at x_axis = 0."""
    shape = (P.n[2], P.n[1], P.n[0])
    c = _centres(P.n[axis], P.dx[axis]) / (P.n[axis] * P.dx[axis])
    side = (c < x0).reshape([-1 if a == axis else 1 for a in (2, 1, 0)])
    side = np.broadcast_to(side, shape)
    rho = np.where(side, left[0], right[0]).astype(np.float64)
    un = np.where(side, left[1], right[1]).astype(np.float64)
    p = np.where(side, left[2], right[2]).astype(np.float64)
    vel = [un if d == axis else np.zeros(shape) for d in range(P.dim)]
    X = [np.ones(shape)] + [np.zeros(shape) for _ in range(P.net.nspec - 1)]
    U = conserved_from(P.gamma, rho, vel, p / rho, X)
    return U


SOD_LEFT = (1.0, 0.0, 1.0)      # (rho, u, p), Sod's shock tube, gamma = 1.4
SOD_RIGHT = (0.125, 0.0, 0.1)


def config_sod(n: int = 128, dim: int = 1, axis: int = 0, nspec: int = 7, seed: int = 0,
               k0: float = 1e3) -> tuple:
    """Sod's shock tube on the unit interval (dim = 1, A -> B with rate
    k0 exp(-10/T), so the shock-heated gas reacts; k0 = 0 leaves it inert) or
    across an n^3 periodic box along `axis` (dim = 3, seeded alpha chain);
    gamma = 1.4, 2 nodes, 2 iterations."""
    if dim == 1:
        net = decay_network(k0=k0)
        P = Problem(dim=1, n=(n, 1, 1), dx=(1.0 / n, 1.0, 1.0), gamma=1.4, net=net, n_nodes=2, n_iters=2)
    else:
        net = alpha_chain(nspec, np.random.default_rng(seed))
        h = 1.0 / n
        P = Problem(dim=3, n=(n, n, n), dx=(h, h, h), gamma=1.4, net=net, n_nodes=2, n_iters=2)
    U = shock_tube_state(P, axis, SOD_LEFT, SOD_RIGHT)
    return P, U.reshape(P.nvar, P.n[2], P.n[1], P.n[0])


def batched_boxes(nbox: int = 200, nspec: int = 7, seed: int = 0,
                  edges=(16, 24, 32, 48, 64), T0: float = 1.0) -> tuple:
    """Ragged batch: per box, edges drawn from `edges` per axis, hot-spot
    amplitude ~ U[1.2, 3] over the background temperature T0; dx = 1/64;
    every box periodic on itself.  The network is drawn first from the same
    seed."""
    rng = np.random.default_rng(seed)
    net = alpha_chain(nspec, rng)
    boxes = []
    for _ in range(nbox):
        e = [int(edges[rng.integers(len(edges))]) for _ in range(3)]
        amp = float(rng.uniform(1.2, 3.0))
        h = 1.0 / 64
        P = Problem(dim=3, n=tuple(e), dx=(h, h, h), gamma=5.0 / 3.0, net=net,
                    n_nodes=3, n_iters=3)
        boxes.append((P, hot_spot_state(P, amp, T0=T0), amp))
    return net, boxes
