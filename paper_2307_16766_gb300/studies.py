"""The paper's benchmark studies (Sec. 4), run on the CUDA path.

Each study sets up the paper's initial fields on the truncated domain and on
a larger periodic domain whose centre crop is the reference (Sec. 4: "fully
periodic LBM simulation on an extended grid"), steps both with the library
and measures the paper's error figures:

  e_Z  = ( sum over the domain of (|Z - Z_ref| / |Z_ref|)^2 )^(1/2)   (Eq. errors)
  ~e_Z = |Z - Z_ref| / |Z_ref|                                       (pointwise)
  R_Z  = I_Z(t2) / I_Z(t1)                                           (Sec. 4.3)

for Z in {rho, u_x, T}.  Everything runs on the GPU (torch tensors from
lbm_get_macros on the device); nothing here changes the method.

  TemperatureStep   Sec. 4.1: a tanh temperature step carried through two
                    artificial sides (periodic top/bottom), D2Q17
  ThermalVortex     Sec. 4.2 / 4.4: a vortex carried out through a
                    characteristic outlet (LODI on the other sides)
  angular_wave      Sec. 4.3: reflection of a plane pulse at angle phi
"""
import math

import numpy as np

from . import Simulation

CS2 = {"D2Q9": 1.0 / 3.0, "D2Q17": 0.3702518670183398497189151, "D2Q37": 0.6979533220196830882384091}
M_OF = {"D2Q9": 1, "D2Q17": 3, "D2Q37": 3}


def _run(lattice, nx, ny, tau, storage="f64", sides=("periodic",) * 4, schemes=("cbc",) * 4,
         viscous="meso", dirichlet="eq", alpha_T=0.0, beta_P=0.0, t_inf=0.0, p_inf=None):
    cs2 = CS2[lattice]
    return {"lattice": lattice, "nx": int(nx), "ny": int(ny), "tau": float(tau), "rho0": 1.0,
            "sides": list(sides), "schemes": list(schemes), "viscous": viscous,
            "dirichlet": dirichlet, "alpha_T": float(alpha_T), "beta_P": float(beta_P),
            "t_inf": float(t_inf), "p_inf": list(p_inf) if p_inf is not None else [cs2] * 4,
            "inflow": [1.0, 0.0, 0.0, 1.0], "storage": storage}


def _macros(sim):
    rho, ux, uy, T = sim.macros(device=True)
    return rho, ux, uy, T


def e_rel(Z, Zref):
    """Eq. errors: (sum ((Z - Z_ref) / Z_ref)^2)^(1/2) over the domain."""
    return float(((Z - Zref) / Zref).pow(2).sum().sqrt())


class _Study:
    """Reference crops recorded every `every` steps; variants compared
    against them."""

    def __init__(self, steps, every):
        self.steps, self.every = steps, every
        self.times = list(range(every, steps + 1, every))
        self.ref = []

    def _record_reference(self, cfg, fields, crop):
        x0, y0, nx, ny = crop
        sim = Simulation(cfg).init_fields(*fields)
        for _ in self.times:
            sim.step(self.every)
            rho, ux, uy, T = _macros(sim)
            self.ref.append(tuple(a[y0:y0 + ny, x0:x0 + nx].clone() for a in (rho, ux, uy, T)))
        sim.close()

    def errors(self, cfg, fields):
        """e_Z(t) for Z = rho, u_x, T at the recorded times (non-finite
        fields give inf from there on)."""
        sim = Simulation(cfg).init_fields(*fields)
        out = {"t": np.array(self.times), "rho": [], "ux": [], "T": []}
        broken = False
        for k in range(len(self.times)):
            if not broken:
                sim.step(self.every)
                try:
                    rho, ux, uy, T = _macros(sim)
                except Exception:
                    broken = True
            if broken:
                for z in ("rho", "ux", "T"):
                    out[z].append(math.inf)
                continue
            r = self.ref[k]
            out["rho"].append(e_rel(rho, r[0]))
            out["ux"].append(e_rel(ux, r[1]))
            out["T"].append(e_rel(T, r[3]))
        sim.close()
        for z in ("rho", "ux", "T"):
            out[z] = np.array(out[z])
        return out


class TemperatureStep(_Study):
    """Sec. 4.1: rho = rho0, u = (Ma c_s, 0), T a smooth step from T0 to T1
    and back (Eq. in Sec. 4.1, read with (tanh + 1) in its second branch so
    that T returns to T0), Lx x Ly = 200 x 20, D2Q17, tau = 0.9, Ma = 0.1,
    T1 = 1.0005, s = 0.5; artificial W/E sides, periodic S/N.  The
    reference is periodic and long enough that no wave re-enters the crop."""

    def __init__(self, steps=1500, every=10, Lx=200, Ly=20, tau=0.9, Ma=0.1, T1=1.0005, s=0.5,
                 lattice="D2Q17", storage="f64"):
        super().__init__(steps, every)
        self.Lx, self.Ly, self.tau, self.lattice, self.storage = Lx, Ly, tau, lattice, storage
        self.u0 = Ma * math.sqrt(CS2[lattice])
        self.T1, self.s = T1, s
        c = math.sqrt(2.0 * CS2[lattice]) + self.u0          # fastest wave speed
        pad = int(c * steps) + 20
        self.Lref = Lx + pad
        self.o = pad // 2
        self._record_reference(_run(lattice, self.Lref, Ly, tau, storage),
                               self.fields(self.Lref, self.o), (self.o, 0, Lx, Ly))

    def fields(self, nx, o):
        Lx, T0, T1, s = self.Lx, 1.0, self.T1, self.s
        xw = np.arange(nx, dtype=np.float64) - o
        T = np.where(xw <= Lx / 2,
                     T1 + (T1 - T0) / 2 * (np.tanh(s * (xw - Lx / 4)) - 1.0),
                     T1 - (T1 - T0) / 2 * (np.tanh(s * (xw - 3 * Lx / 4)) + 1.0))
        T = np.tile(T, (self.Ly, 1))
        return (np.ones_like(T), np.full_like(T, self.u0), np.zeros_like(T), T)

    VARIANTS = {
        "zg": dict(sides=("zg", "zg", "periodic", "periodic")),
        "lodi": dict(sides=("cbc", "cbc", "periodic", "periodic"), schemes=("lodi",) * 4),
        "lodi_neep": dict(sides=("cbc", "cbc", "periodic", "periodic"), schemes=("lodi",) * 4,
                          dirichlet="neep"),
        "cbc": dict(sides=("cbc", "cbc", "periodic", "periodic"), schemes=("cbc",) * 4),
        "cbc_neep": dict(sides=("cbc", "cbc", "periodic", "periodic"), schemes=("cbc",) * 4,
                         dirichlet="neep"),
    }

    def run(self, variant):
        cfg = _run(self.lattice, self.Lx, self.Ly, self.tau, self.storage, **self.VARIANTS[variant])
        return self.errors(cfg, self.fields(self.Lx, 0))


class ThermalVortex(_Study):
    """Sec. 4.2: Lx x Ly = 150 x 150, normalised coordinates
    x^ = 2 (x - 1) / (Lx - 1) - 1 (x counted from 1), a vortex at
    (x^0, 0) = (K / (Lx - 1), 0) (K = 0: the paper leaves K open) of radius
    r^ = 0.7 and strength b = 3/20 in a stream u0 = (Ma c_s, 0), Ma = 0.1:
    u = u0 + (5 c_s Ma / 2) 2^(-(x^2 + y^2) / b^2) (y, -x) and
    T = T0 + y^ (5 c_s Ma / 2) 2^(-(x^2 + y^2) / b^2) inside r^ (as
    printed).  The outlet (E side) takes the scheme under study, the other
    sides LODI, the corners LODI; alpha = Ma, beta = 0, T_inf = 0 for the
    relaxed schemes.  isothermal=True gives the iso-thermal vortex of
    Sec. 4.4 (T = T0)."""

    def __init__(self, steps=1200, every=10, L=150, nu=0.1, Ma=0.1, r=0.7, b=0.15, K=0.0,
                 lattice="D2Q17", storage="f64", isothermal=False, ref_side=None):
        super().__init__(steps, every)
        self.L, self.lattice, self.storage, self.Ma = L, lattice, storage, Ma
        self.r, self.b, self.K, self.isothermal = r, b, K, isothermal
        cs2 = CS2[lattice]
        self.cs = math.sqrt(cs2)
        self.tau = 0.5 + nu / cs2
        c = (math.sqrt(2.0 * cs2) if lattice != "D2Q9" else self.cs) + Ma * self.cs
        self.Lref = ref_side or (L + int(c * steps) + 20)
        self.o = (self.Lref - L) // 2
        self._record_reference(_run(lattice, self.Lref, self.Lref, self.tau, storage),
                               self.fields(self.Lref, self.o), (self.o, self.o, L, L))

    def fields(self, n, o):
        L, Ma, cs = self.L, self.Ma, self.cs
        i = np.arange(n, dtype=np.float64) - o
        xh = 2.0 * i / (L - 1) - 1.0
        X, Y = np.meshgrid(xh, xh)
        x0 = self.K / (L - 1)
        dx, dy = X - x0, Y
        inside = dx * dx + dy * dy < self.r * self.r
        amp = 2.5 * cs * Ma * np.power(2.0, -(dx * dx + dy * dy) / (self.b * self.b))
        ux = Ma * cs + np.where(inside, amp * dy, 0.0)
        uy = np.where(inside, -amp * dx, 0.0)
        T = np.ones_like(X) if self.isothermal else 1.0 + np.where(inside, Y * amp, 0.0)
        return (np.ones_like(X), ux, uy, T)

    def config(self, outlet="cbc_relax", alpha=None, dirichlet="eq", viscous="meso", zg=False):
        if zg:
            return _run(self.lattice, self.L, self.L, self.tau, self.storage, sides=("zg",) * 4,
                        viscous=viscous)
        a = self.Ma if alpha is None else alpha
        return _run(self.lattice, self.L, self.L, self.tau, self.storage, sides=("cbc",) * 4,
                    schemes=("lodi", outlet, "lodi", "lodi"), viscous=viscous, dirichlet=dirichlet,
                    alpha_T=a, beta_P=0.0, t_inf=0.0)

    def run(self, **kw):
        return self.errors(self.config(**kw), self.fields(self.L, 0))

    def pointwise(self, step, **kw):
        """~e_Z at one step (a multiple of `every`) for rho and u_x."""
        cfg = self.config(**kw)
        sim = Simulation(cfg).init_fields(*self.fields(self.L, 0))
        sim.step(step)
        rho, ux, uy, T = _macros(sim)
        sim.close()
        r = self.ref[step // self.every - 1]
        return ((rho - r[0]).abs() / r[0].abs()).cpu().numpy(), ((ux - r[1]).abs() / r[1].abs()).cpu().numpy()


def angular_wave(phi, variants=("zg", "lodi", "cbc"), Lx=200, Ly=700, nu=0.1, s=1.0 / 50,
                 lattice="D2Q17", storage="f64"):
    """Sec. 4.3: rho = rho0, u = 0, T = T0 + 0.1 exp(-x^2 / (2 s^2)) with
    x^ = (cos phi, sin phi) . (x, y) in coordinates centred on the domain and
    scaled by (Lx - 1) / 2 along both axes (so phi is the geometric angle);
    artificial W/E sides, periodic S/N, Lx x Ly = 200 x 700, nu = 0.1.
    R_rho = I(t2) / I(t1) along the midline y = Ly / 2: I(t1) the incident
    amplitude max |rho - rho0| of the reference over the left half before
    the pulse reaches the W side, I(t2) = max |rho - rho_ref| over the left
    half once the reflection is back inside (rho_ref: a 4x longer periodic
    run).  Returns {variant: R_rho}."""
    cs2 = CS2[lattice]
    tau = 0.5 + nu / cs2
    c = math.sqrt(2.0 * cs2) if lattice != "D2Q9" else math.sqrt(cs2)
    M = M_OF[lattice]
    ph = math.radians(phi)
    scale = (Lx - 1) / 2.0

    def fields(nx, o):
        x = (np.arange(nx, dtype=np.float64) - o - (Lx - 1) / 2.0) / scale
        y = (np.arange(Ly, dtype=np.float64) - (Ly - 1) / 2.0) / scale
        X, Y = np.meshgrid(x, y)
        xh = math.cos(ph) * X + math.sin(ph) * Y
        T = 1.0 + 0.1 * np.exp(-xh * xh / (2.0 * s * s))
        return (np.ones_like(T), np.zeros_like(T), np.zeros_like(T), T)

    # time for the pulse to cross from the centre to the W side along the
    # midline (normal speed c, normal distance (Lx/2) cos phi)
    t_hit = (Lx / 2.0 - M) * math.cos(ph) / c
    t1 = int(0.5 * t_hit)
    t2 = int(2.0 * t_hit) + 10
    o = (4 * Lx - Lx) // 2
    mid = Ly // 2
    ref = Simulation(_run(lattice, 4 * Lx, Ly, tau, storage)).init_fields(*fields(4 * Lx, o))
    ref.step(t1)
    r1 = _macros(ref)[0][mid, o:o + Lx // 2]
    inc = float((r1 - 1.0).abs().max())
    ref.step(t2 - t1)
    r2 = _macros(ref)[0][mid, o:o + Lx]
    ref.close()
    sides = {"zg": dict(sides=("zg", "zg", "periodic", "periodic")),
             "lodi": dict(sides=("cbc", "cbc", "periodic", "periodic"), schemes=("lodi",) * 4),
             "cbc": dict(sides=("cbc", "cbc", "periodic", "periodic"), schemes=("cbc",) * 4)}
    out = {}
    for v in variants:
        sim = Simulation(_run(lattice, Lx, Ly, tau, storage, **sides[v])).init_fields(*fields(Lx, 0))
        sim.step(t2)
        rho = _macros(sim)[0][mid, :]
        sim.close()
        out[v] = float((rho[: Lx // 2] - r2[: Lx // 2]).abs().max()) / inc
    return out
