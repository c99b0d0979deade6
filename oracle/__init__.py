"""ctypes wrapper of the plain FP64 CPU oracle (sdc_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "sdc_oracle.c")

MAX_SPEC = 32
MAX_REAC = 32

NEWTON_OK, NEWTON_MAXIT, NEWTON_NONPHYSICAL, NEWTON_SINGULAR = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP over zones)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "sdc_oracle.h"))):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-fopenmp", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3), ("gamma", C.c_double),
        ("limiter", C.c_int), ("nspec", C.c_int), ("nreac", C.c_int), ("rate_law", C.c_int),
        ("mass", C.c_double * MAX_SPEC), ("a", C.c_double * MAX_REAC), ("nu", C.c_double * MAX_REAC),
        ("Q", C.c_double * MAX_REAC), ("reac", (C.c_int * 2) * MAX_REAC), ("cnt", (C.c_int * 2) * MAX_REAC),
        ("prod", C.c_int * MAX_REAC), ("n_nodes", C.c_int), ("n_iters", C.c_int),
        ("newton_rtol", C.c_double), ("newton_maxit", C.c_int), ("node_type", C.c_int),
        ("split_op", C.c_int), ("space_order", C.c_int),
    ]


NODE_TYPES = {"lobatto": 0, "radau": 1}


class _Stats(C.Structure):
    _fields_ = [("newton_iters_total", C.c_longlong), ("newton_solves", C.c_longlong),
                ("n_fail", C.c_longlong), ("hist", C.c_longlong * 64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        pp = C.POINTER(_Problem)
        _lib.orc_nvar.argtypes = [pp]
        _lib.orc_quad_weights.argtypes = [C.c_int, C.c_int, dp]
        _lib.orc_nodes.argtypes = [C.c_int, C.c_int, dp]
        _lib.orc_temperature.argtypes = [pp, C.c_double, dp, C.c_double]
        _lib.orc_temperature.restype = C.c_double
        _lib.orc_advective.argtypes = [pp, dp, dp]
        _lib.orc_advective_term.argtypes = [pp, dp, dp]
        _lib.orc_reaction_source4.argtypes = [pp, dp, dp]
        _lib.orc_limited_faces.argtypes = [pp, C.c_int, dp, dp, dp, dp]
        _lib.orc_avg_to_point.argtypes = [pp, C.c_int, dp, dp]
        _lib.orc_point_to_avg.argtypes = [pp, C.c_int, dp, dp]
        _lib.orc_hllc.argtypes = [pp, C.c_int, dp, dp, dp]
        _lib.orc_hllc_star.argtypes = [pp, C.c_int, dp, dp, dp, dp, dp]
        _lib.orc_rates.argtypes = [pp, C.c_double, dp, dp, dp, dp]
        _lib.orc_reaction_source.argtypes = [pp, dp, dp]
        _lib.orc_newton_zone.argtypes = [pp, C.c_double, dp, dp, C.c_double, dp, ip]
        _lib.orc_react_newton.argtypes = [pp, dp, C.c_double, dp, dp, ip, ip, C.POINTER(_Stats)]
        _lib.orc_node_integral.argtypes = [pp, C.POINTER(dp), C.POINTER(dp), C.c_double, C.c_int, dp]
        _lib.orc_sdc_step.argtypes = [pp, dp, C.c_double, C.POINTER(_Stats)]
        _lib.orc_strang_step.argtypes = [pp, dp, C.c_double, C.POINTER(_Stats)]
        _lib.orc_sdc_step_nodes.argtypes = [pp, dp, C.c_double, C.POINTER(_Stats), dp]
        _lib.orc_cfl_dt.argtypes = [pp, dp, C.c_double]
        _lib.orc_cfl_dt.restype = C.c_double
    return _lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_int))


class Oracle:
    """The oracle bound to one problem (box, network, SDC parameters)."""

    def __init__(self, P):
        self.P = P
        s = _Problem()
        s.dim = P.dim
        for d in range(3):
            s.n[d] = int(P.n[d])
            s.dx[d] = float(P.dx[d])
        s.gamma = P.gamma
        s.limiter = P.limiter
        net = P.net
        s.nspec, s.nreac, s.rate_law = net.nspec, net.nreac, net.rate_law
        for i in range(net.nspec):
            s.mass[i] = float(net.mass[i])
        for j in range(net.nreac):
            s.a[j], s.nu[j], s.Q[j] = float(net.a[j]), float(net.nu[j]), float(net.Q[j])
            for k in range(2):
                s.reac[j][k] = int(net.reac[j][k])
                s.cnt[j][k] = int(net.cnt[j][k])
            s.prod[j] = int(net.prod[j])
        s.n_nodes, s.n_iters = P.n_nodes, P.n_iters
        s.newton_rtol, s.newton_maxit = P.newton_rtol, P.newton_maxit
        s.node_type = NODE_TYPES[P.nodes]
        s.split_op = 0
        s.space_order = int(P.space_order)
        self.s = s
        self.L = lib()
        self.nvar = P.nvar
        self.N = P.nzones
        self.n = net.nspec + 1

    def _flat(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.size == self.nvar * self.N
        return U

    def advective(self, U):
        """A(U) of the problem's spatial order (PLM/HLLC, or the fourth-order operator)."""
        U = self._flat(U)
        A = np.empty_like(U)
        self.L.orc_advective_term(C.byref(self.s), _dp(U), _dp(A))
        return A

    def reaction_source(self, U):
        """R on zone averages (second order) or the averaged source of the fourth-order scheme."""
        U = self._flat(U)
        R = np.empty((self.n,) + U.shape[1:])
        if self.P.space_order == 4:
            self.L.orc_reaction_source4(C.byref(self.s), _dp(U), _dp(R))
        else:
            self.L.orc_reaction_source(C.byref(self.s), _dp(U), _dp(R))
        return R

    def avg_to_point(self, F):
        """Zone-centre values from zone averages, f - L f / 24 (fields first)."""
        F = np.ascontiguousarray(F, dtype=np.float64)
        out = np.empty_like(F)
        self.L.orc_avg_to_point(C.byref(self.s), int(F.shape[0]), _dp(F), _dp(out))
        return out

    def point_to_avg(self, F):
        """Zone averages from zone-centre values, f + L f / 24 (fields first)."""
        F = np.ascontiguousarray(F, dtype=np.float64)
        out = np.empty_like(F)
        self.L.orc_point_to_avg(C.byref(self.s), int(F.shape[0]), _dp(F), _dp(out))
        return out

    def limited_faces(self, direction, Wa, Wf):
        """The fourth-order form's limited face states from averaged primitives Wa
        and face values Wf ([nvar][...]): WL (upper face of each zone) and WR (at
        zone z: the lower face of zone z+1)."""
        Wa = np.ascontiguousarray(Wa, dtype=np.float64)
        Wf = np.ascontiguousarray(Wf, dtype=np.float64)
        WL, WR = np.empty_like(Wa), np.empty_like(Wa)
        self.L.orc_limited_faces(C.byref(self.s), int(direction), _dp(Wa), _dp(Wf), _dp(WL), _dp(WR))
        return WL, WR

    def rates(self, rho, mom, w, jac=True):
        mom = np.ascontiguousarray(np.atleast_1d(mom), dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        R = np.empty(self.n)
        J = np.empty((self.n, self.n)) if jac else None
        self.L.orc_rates(C.byref(self.s), float(rho), _dp(mom), _dp(w), _dp(R),
                         _dp(J) if jac else None)
        return (R, J) if jac else R

    def hllc(self, direction, qL, qR):
        qL = np.ascontiguousarray(qL, dtype=np.float64)
        qR = np.ascontiguousarray(qR, dtype=np.float64)
        F = np.empty(self.nvar)
        self.L.orc_hllc(C.byref(self.s), int(direction), _dp(qL), _dp(qR), _dp(F))
        return F

    def hllc_star(self, direction, qL, qR):
        """Wave speeds (S_L, S*, S_R) and the star states U*_L, U*_R (mass,
        momenta, energy) of the HLLC fan between two primitive states."""
        qL = np.ascontiguousarray(qL, dtype=np.float64)
        qR = np.ascontiguousarray(qR, dtype=np.float64)
        S = np.empty(3)
        UsL = np.empty(2 + self.P.dim)
        UsR = np.empty(2 + self.P.dim)
        self.L.orc_hllc_star(C.byref(self.s), int(direction), _dp(qL), _dp(qR), _dp(S), _dp(UsL), _dp(UsR))
        return S, UsL, UsR

    def temperature(self, rho, mom, rhoE):
        mom = np.ascontiguousarray(np.atleast_1d(mom), dtype=np.float64)
        return self.L.orc_temperature(C.byref(self.s), float(rho), _dp(mom), float(rhoE))

    def newton_zone(self, rho, mom, rhs_w, dt_m, guess):
        mom = np.ascontiguousarray(np.atleast_1d(mom), dtype=np.float64)
        rhs_w = np.ascontiguousarray(rhs_w, dtype=np.float64)
        w = np.array(guess, dtype=np.float64)
        it = C.c_int(0)
        st = self.L.orc_newton_zone(C.byref(self.s), float(rho), _dp(mom), _dp(rhs_w), float(dt_m),
                                    _dp(w), C.byref(it))
        return w, st, it.value

    def react_newton(self, rhs, dt_m, guess):
        """Returns (U_new, R_new, zone_status, zone_iters, stats)."""
        rhs = self._flat(rhs)
        U = np.array(self._flat(guess), copy=True)
        R = np.empty((self.n,) + U.shape[1:])
        zs = np.empty(U.shape[1:], dtype=np.int32)
        zi = np.empty(U.shape[1:], dtype=np.int32)
        st = _Stats()
        self.L.orc_react_newton(C.byref(self.s), _dp(rhs), float(dt_m), _dp(U), _dp(R), _ip(zs), _ip(zi),
                                C.byref(st))
        return U, R, zs, zi, st

    def node_integral(self, A_nodes, R_nodes, dt, m):
        A_nodes = [self._flat(a) for a in A_nodes]
        R_nodes = [np.ascontiguousarray(r, dtype=np.float64) for r in R_nodes]
        Ap = (C.POINTER(C.c_double) * len(A_nodes))(*[_dp(a) for a in A_nodes])
        Rp = (C.POINTER(C.c_double) * len(R_nodes))(*[_dp(r) for r in R_nodes])
        I = np.empty_like(A_nodes[0])
        self.L.orc_node_integral(C.byref(self.s), Ap, Rp, float(dt), int(m), _dp(I))
        return I

    def step(self, U, dt, nodes=False):
        U = np.array(self._flat(U), copy=True)
        st = _Stats()
        if nodes:
            out = np.empty((self.P.n_nodes,) + U.shape)
            rc = self.L.orc_sdc_step_nodes(C.byref(self.s), _dp(U), float(dt), C.byref(st), _dp(out))
            assert rc == 0
            return U, st, out
        rc = self.L.orc_sdc_step(C.byref(self.s), _dp(U), float(dt), C.byref(st))
        assert rc == 0
        return U, st

    def strang_step(self, U, dt):
        """Strang-split baseline: reactions dt/2, advection dt, reactions dt/2,
        each by this problem's SDC step with the other operator off."""
        U = np.array(self._flat(U), copy=True)
        st = _Stats()
        rc = self.L.orc_strang_step(C.byref(self.s), _dp(U), float(dt), C.byref(st))
        assert rc == 0
        return U, st

    def cfl_dt(self, U, cfl=None):
        U = self._flat(U)
        return self.L.orc_cfl_dt(C.byref(self.s), _dp(U), float(self.P.cfl if cfl is None else cfl))

    def run(self, U, nsteps, dts=None):
        """nsteps SDC steps with the CFL dt (or the given dt sequence);
        returns (U, list of dt, stats list)."""
        U = self._flat(U)
        dt_used, stats = [], []
        for s in range(nsteps):
            dt = self.cfl_dt(U) if dts is None else dts[s]
            U, st = self.step(U, dt)
            dt_used.append(dt)
            stats.append(st)
        return U, dt_used, stats


def quad_weights(M, nodes="lobatto"):
    q = np.zeros((M - 1) * M)
    rc = lib().orc_quad_weights(NODE_TYPES[nodes], int(M), _dp(q))
    assert rc == 0
    return q.reshape(M - 1, M)


def nodes(M, nodes="lobatto"):
    tau = np.zeros(M)
    rc = lib().orc_nodes(NODE_TYPES[nodes], int(M), _dp(tau))
    assert rc == 0
    return tau
