"""ctypes binding of the plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py``.  The product package never
imports it, and the oracle shares no code with the CUDA path.

A run is described by a plain dict (see ``lbm_workloads``) with the keys
``lattice`` ("D2Q9" | "D2Q37" | "D2Q17"), ``nx``, ``ny``, ``tau``, ``rho0``, ``sides``
(four of "periodic" | "cbc" | "inflow" | "zg", order W, E, S, N),
``schemes`` (four of "lodi" | "lodi_relax" | "cbc" | "cbc_relax"),
``viscous`` ("meso" | "fd" | "off"), ``dirichlet`` ("eq" | "neep" | "reg"), ``alpha_T``, ``beta_P``,
``t_inf``, ``p_inf`` (four values), ``inflow`` (rho, ux, uy, T), ``alpha_V`` (the relaxation of
the viscous term in Eq. CBC-Relax, 0 by default: the paper's equation) and, for tests only,
``meso_depth`` (where the mesoscopic viscous stencil starts below x_f; default M).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

LATTICES = {"D2Q9": 0, "D2Q37": 1, "D2Q17": 2}
SIDES = {"periodic": 0, "cbc": 1, "inflow": 2, "zg": 3}
SCHEMES = {"lodi": 0, "lodi_relax": 1, "cbc": 2, "cbc_relax": 3}
DIRICHLET = {"eq": 0, "neep": 1, "reg": 2}
VISCOUS = {"meso": 0, "fd": 1, "off": 2}


class Params(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("tau", C.c_double), ("rho0", C.c_double),
        ("side", C.c_int * 4), ("scheme", C.c_int * 4),
        ("viscous", C.c_int), ("dirichlet", C.c_int),
        ("alpha_T", C.c_double), ("beta_P", C.c_double), ("t_inf", C.c_double),
        ("p_inf", C.c_double * 4), ("inflow", C.c_double * 4),
        ("alpha_V", C.c_double), ("meso_depth", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_lattice_info.argtypes = [C.c_int, ip, ip, dp, ip, dp]
        L.orc_feq.argtypes = [C.c_int, C.c_double, dp, dp]
        L.orc_regularize.argtypes = [C.c_int, dp]
        L.orc_moments.argtypes = [C.c_int, C.c_double, dp, dp]
        L.orc_char_matrices.argtypes = [C.c_int, C.c_double, dp, dp, dp, dp]
        L.orc_char_rhs.argtypes = [C.POINTER(Params), dp, dp, dp, dp, C.c_int, C.c_double, C.c_int, dp]
        L.orc_corner_rhs.argtypes = [C.POINTER(Params), C.c_int, dp, dp, dp, dp]
        L.orc_rk4_scalar.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
        L.orc_rk4_scalar.restype = C.c_double
        L.orc_create.argtypes = [C.POINTER(Params)]
        L.orc_create.restype = C.c_void_p
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_init.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_macros.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.orc_populations.argtypes = [C.c_void_p, dp]
        L.orc_neq_moments.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        L.orc_vis_meso_at.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, dp]
        L.orc_boundary_state.argtypes = [C.c_void_p, dp]
        L.orc_steps_done.argtypes = [C.c_void_p]
        L.orc_steps_done.restype = C.c_long
        L.orc_threads.restype = C.c_int
        L.orc_set_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(cfg) -> Params:
    p = Params()
    p.lattice = LATTICES[cfg["lattice"]]
    p.nx, p.ny = int(cfg["nx"]), int(cfg["ny"])
    p.tau = float(cfg["tau"])
    p.rho0 = float(cfg.get("rho0", 1.0))
    for i, s in enumerate(cfg.get("sides", ["periodic"] * 4)):
        p.side[i] = SIDES[s]
    for i, s in enumerate(cfg.get("schemes", ["cbc"] * 4)):
        p.scheme[i] = SCHEMES[s]
    p.viscous = VISCOUS[cfg.get("viscous", "meso")]
    p.dirichlet = DIRICHLET[cfg.get("dirichlet", "eq")]
    p.alpha_T = float(cfg.get("alpha_T", 0.0))
    p.beta_P = float(cfg.get("beta_P", 0.0))
    p.t_inf = float(cfg.get("t_inf", 0.0))
    p.alpha_V = float(cfg.get("alpha_V", 0.0))
    p.meso_depth = int(cfg.get("meso_depth", -1))
    cs2 = lattice_info(cfg["lattice"])["cs2"]
    pinf = cfg.get("p_inf", [cs2 * p.rho0] * 4)
    for i in range(4):
        p.p_inf[i] = float(pinf[i])
    inflow = cfg.get("inflow", [p.rho0, 0.0, 0.0, 1.0])
    for i in range(4):
        p.inflow[i] = float(inflow[i])
    return p


def lattice_info(name):
    L = lib()
    q = C.c_int()
    M = C.c_int()
    cs2 = C.c_double()
    c = (C.c_int * 74)()
    w = (C.c_double * 37)()
    if L.orc_lattice_info(LATTICES[name], C.byref(q), C.byref(M), C.byref(cs2), c, w):
        raise ValueError(name)
    n = q.value
    return {"q": n, "M": M.value, "cs2": cs2.value,
            "c": np.array(c[: 2 * n], dtype=np.int64).reshape(n, 2),
            "w": np.array(w[:n], dtype=np.float64)}


def feq(lattice, rho0, U):
    """Shifted equilibrium f^eq - w rho0 at U = (drho, ux, uy, dT)."""
    info = lattice_info(lattice)
    g = np.zeros(info["q"])
    u = _f64(U)
    lib().orc_feq(LATTICES[lattice], rho0, _dp(u), _dp(g))
    return g


def regularize(lattice, g):
    """Hermite projection (orders 2, and 3 on the thermal lattices) of a
    non-equilibrium vector g; returns a new array."""
    out = _f64(g).copy()
    lib().orc_regularize(LATTICES[lattice], _dp(out))
    return out


def moments(lattice, rho0, g):
    """(drho, ux, uy, dT) of shifted populations g."""
    g = _f64(g)
    U = np.zeros(4)
    lib().orc_moments(LATTICES[lattice], rho0, _dp(g), _dp(U))
    return U


def char_matrices(lattice, rho0, Ul):
    S = np.zeros(16)
    Si = np.zeros(16)
    lam = np.zeros(4)
    u = _f64(Ul)
    lib().orc_char_matrices(LATTICES[lattice], rho0, _dp(u), _dp(S), _dp(Si), _dp(lam))
    n = 3 if lattice == "D2Q9" else 4
    return S.reshape(4, 4)[:n, :n], Si.reshape(4, 4)[:n, :n], lam[:n]


def char_rhs(cfg, Ul, dUn, TT, VV, mask, dP, scheme):
    p = make_params(cfg)
    k = np.zeros(4)
    args = [_f64(a) for a in (Ul, dUn, TT, VV)]
    lib().orc_char_rhs(C.byref(p), *[_dp(a) for a in args], int(mask), float(dP),
                       SCHEMES[scheme], _dp(k))
    return k


def corner_rhs(cfg, cid, Uc, U1, U2):
    """Lab-frame right-hand side of corner cid from the corner node's state
    and those one and two diagonal steps inward (deviation form)."""
    p = make_params(cfg)
    k = np.zeros(4)
    args = [_f64(a) for a in (Uc, U1, U2)]
    if lib().orc_corner_rhs(C.byref(p), int(cid), *[_dp(a) for a in args], _dp(k)):
        raise ValueError("bad corner")
    return k


def rk4_scalar(lam, y0, h, nsteps):
    return lib().orc_rk4_scalar(lam, y0, h, nsteps)


def threads():
    return lib().orc_threads()


def set_threads(n):
    """Threads of the following steps; returns the count now in use."""
    return lib().orc_set_threads(int(n))


class Sim:
    """One oracle run: ``Sim(cfg).init(rho, ux, uy, T).step(n).macros()``."""

    def __init__(self, cfg):
        self.cfg = dict(cfg)
        self._p = make_params(cfg)
        self._h = lib().orc_create(C.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.nx, self.ny = self._p.nx, self._p.ny
        self.q = lattice_info(cfg["lattice"])["q"]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init(self, rho, ux, uy, T):
        shape = (self.ny, self.nx)
        arrs = [_f64(np.broadcast_to(a, shape)) for a in (rho, ux, uy, T)]
        lib().orc_init(self._h, *[_dp(a) for a in arrs])
        return self

    def step(self, n=1):
        lib().orc_step(self._h, int(n))
        return self

    @property
    def steps_done(self):
        return lib().orc_steps_done(self._h)

    def macros(self):
        """(rho, ux, uy, T), each [ny, nx] float64."""
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        lib().orc_macros(self._h, *[_dp(a) for a in out])
        return tuple(out)

    def populations(self):
        g = np.zeros((self.ny, self.nx, self.q))
        lib().orc_populations(self._h, _dp(g))
        return g

    def neq_moments(self, x, y):
        out = np.zeros(5)
        lib().orc_neq_moments(self._h, int(x), int(y), _dp(out))
        return out

    def vis_meso_at(self, side, x, y):
        V = np.zeros(4)
        lib().orc_vis_meso_at(self._h, int(side), int(x), int(y), _dp(V))
        return V

    def boundary_state(self):
        U = np.zeros((self.ny, self.nx, 4))
        lib().orc_boundary_state(self._h, _dp(U))
        return U


# ------------------------------------------------------ pressure loss -------
# The loss used to tune the relaxation parameters: the squared deviation of
# the pressure P = rho c_s^2 T (isothermal: rho c_s^2) from a reference over
# the nodes off the M boundary layers, summed over the steps -- the
# reflection measure of Sec. "Numerical Results" (pressure against a
# reference run on a larger domain) taken as an energy.  Here P - c_s^2 rho0
# is formed as c_s^2 ((rho - rho0) + rho0 (T - 1) + (rho - rho0)(T - 1)).

def pressure_loss(cfg, fields, steps, dP_ref=None):
    """J = sum_{n=1..steps} sum_x (P_n(x) - c_s^2 rho0 - dP_ref[n-1](x))^2
    over x off the boundary layers of non-periodic axes.  dP_ref: None or
    an array [steps, ny, nx]."""
    info = lattice_info(cfg["lattice"])
    cs2, M = info["cs2"], info["M"]
    rho0 = cfg.get("rho0", 1.0)
    nx, ny = cfg["nx"], cfg["ny"]
    perx = cfg["sides"][0] == "periodic"
    pery = cfg["sides"][2] == "periodic"
    xs = slice(0, nx) if perx else slice(M, nx - M)
    ys = slice(0, ny) if pery else slice(M, ny - M)
    s = Sim(cfg).init(*fields)
    J = 0.0
    for n in range(steps):
        s.step(1)
        rho, ux, uy, T = s.macros()
        dr = rho - rho0
        dP = cs2 * (dr + rho0 * (T - 1.0) + dr * (T - 1.0)) if cfg["lattice"] != "D2Q9" else cs2 * dr
        e = dP[ys, xs] - (0.0 if dP_ref is None else dP_ref[n][ys, xs])
        J += float(np.sum(e * e))
    return J


def _value_of(cfg, name):
    return cfg["p_inf"][0] if name == "p_inf" else cfg.get(name, 0.0)


def _with_value(cfg, name, v):
    c = dict(cfg)
    c[name] = [float(v)] * 4 if name == "p_inf" else float(v)
    return c


def pressure_loss_fd_gradient(cfg, fields, steps, h=(1e-4, 1e-4, 1e-4), dP_ref=None,
                              params=("alpha_T", "beta_P", "p_inf")):
    """Central differences of pressure_loss in the named relaxation
    parameters (any of alpha_T, beta_P, p_inf, alpha_V, t_inf), step h[k]
    for params[k]; p_inf is moved on every side together (cfg's p_inf must
    be equal on all sides)."""
    g = []
    for name, hk in zip(params, h):
        v = _value_of(cfg, name)
        Jp = pressure_loss(_with_value(cfg, name, v + hk), fields, steps, dP_ref)
        Jm = pressure_loss(_with_value(cfg, name, v - hk), fields, steps, dP_ref)
        g.append((Jp - Jm) / (2.0 * hk))
    return g
