"""Helpers shared by the GPU parity tests (tests only)."""
import numpy as np

import oracle as O


def rel_err(gpu, orc, nvar, dim, species_floor=None):
    """Per-field relative infinity-norm error |gpu - orc|_inf / |orc|_inf,
    every field against its own largest oracle value (floor 1e-30), species
    included.  With species_floor set, species fields are instead taken
    relative to max(|rho X_i|_inf, species_floor * |rho|_inf)."""
    g = np.asarray(gpu).reshape(nvar, -1)
    o = np.asarray(orc).reshape(nvar, -1)
    rho_max = np.abs(o[0]).max()
    out = []
    for f in range(nvar):
        den = max(np.abs(o[f]).max(), 1e-30)
        if f >= 2 + dim and species_floor is not None:
            den = max(den, species_floor * rho_max)
        out.append(np.abs(g[f] - o[f]).max() / den)
    return np.array(out)


def flux_term_scale(U, P):
    """Per field, a bound on the terms whose difference over dx is the
    advective term: the HLLC flux combines F(U) and S U, each at most
    (|U_f| + p) (|u| + c) per field (p only in the momenta and the energy),
    over the smallest dx.  A's rounding error is a small multiple of the unit
    round-off times this, whatever the size of A itself."""
    V = np.asarray(U).reshape(P.nvar, -1)
    dim = P.dim
    rho = V[0]
    u = V[1:1 + dim] / rho
    ke = 0.5 * rho * (u * u).sum(0)
    p = (P.gamma - 1.0) * (V[1 + dim] - ke)
    c = np.sqrt(P.gamma * np.maximum(p, 0.0) / rho)
    speed = (np.abs(u).max(0) + c).max()
    pmax = np.abs(p).max()
    idx = 1.0 / min(P.dx[:dim])
    out = []
    for f in range(P.nvar):
        extra = pmax if 1 <= f <= 1 + dim else 0.0
        out.append((np.abs(V[f]).max() + extra) * speed * idx)
    return np.array(out)


def rel_err_R(gpu, orc, n, scale):
    g = np.asarray(gpu).reshape(n, -1)
    o = np.asarray(orc).reshape(n, -1)
    return np.array([np.abs(g[r] - o[r]).max() / max(np.abs(o[r]).max(), scale) for r in range(n)])


def newton_guess(o, rhs, Rk, dtm, prev):
    """The sweep's Newton start, as the oracle forms it: the explicit predictor
    rhs + dt_m R^{m+1,(k)} in the reactive fields where it has a positive
    temperature and no mass fraction below -0.01, the previous iterate prev
    elsewhere."""
    P = o.P
    dim = P.dim
    g = rhs.copy()
    g[1 + dim:] = rhs[1 + dim:] + dtm * Rk
    G = g.reshape(P.nvar, -1)
    ke = 0.5 * (G[1:1 + dim] ** 2).sum(0) / G[0]
    ok = (G[1 + dim] - ke) > 0
    ok &= ~(G[2 + dim:] < -1e-2 * G[0]).any(0)
    out = prev.reshape(P.nvar, -1).copy()
    out[:, ok] = G[:, ok]
    return out.reshape(rhs.shape)


def oracle_sweep_inputs(o, U, dt, k_iters=1, m_target=None, predictor=True):
    """Run the oracle sweep in Python from its building blocks and return the
    (rhs, guess, dt_m) seen by the Newton solve at the last (k, m) visited.
    predictor=False: the guess is the previous iterate, the start of the
    FP32-Jacobian solves (the oracle's own sweep takes the predictor)."""
    P = o.P
    M = P.n_nodes
    dim = P.dim
    tau = [0.0, 1.0] if M == 2 else [0.0, 0.5, 1.0]
    Un = [U.copy() for _ in range(M)]
    A0 = o.advective(U)
    R0 = o.reaction_source(U)
    Aold = [A0] * M
    Rold = [R0] * M
    last = None
    for k in range(k_iters):
        Anew = [A0] + [None] * (M - 1)
        Rnew = [R0] + [None] * (M - 1)
        for m in range(M - 1):
            dtm = dt * (tau[m + 1] - tau[m])
            Anew[m] = A0 if m == 0 else o.advective(Un[m])
            I = o.node_integral(Aold, Rold, dt, m)
            rhs = Un[m] + dtm * (Anew[m] - Aold[m])
            rhs[1 + dim:] -= dtm * Rold[m + 1]
            rhs = rhs + I
            guess = newton_guess(o, rhs, Rold[m + 1], dtm, Un[m + 1]) if predictor else Un[m + 1]
            last = (rhs.copy(), guess.copy(), dtm)
            if m_target is not None and m == m_target and k == k_iters - 1:
                return last
            Unew, Rn, zs, zi, st = o.react_newton(rhs, dtm, newton_guess(o, rhs, Rold[m + 1], dtm, Un[m + 1]))
            Un[m + 1] = Unew
            Rnew[m + 1] = Rn
        if k < k_iters - 1:
            Anew[M - 1] = o.advective(Un[M - 1])
        Aold, Rold = Anew, Rnew
    return last
