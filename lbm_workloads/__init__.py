"""Seeded synthetic workloads: run descriptions and initial fields.

This module holds no arithmetic of the method itself.  It only builds the
inputs that both the CUDA path and the CPU oracle receive: a run description
(plain dict) and initial macroscopic fields (rho, ux, uy, T) as float64
arrays of shape [ny, nx].  Random draws come from SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so a
seed names the same inputs on every machine.

The initial fields follow the shapes of the paper's own benchmarks (Sec. 4):
Gaussian acoustic / thermal pulses, a vortex convected by a uniform stream
(here the classical isentropic vortex), plane shear and temperature waves.
"""
import math

import numpy as np

# Lattice sound speeds squared (Appendix B), used only to scale inputs:
# background velocity Ma * c_s and the default target pressure rho0 c_s^2.
CS2 = {"D2Q9": 1.0 / 3.0, "D2Q37": 0.6979533220196830882384091,
       "D2Q17": 0.3702518670183398497189151}
M_OF = {"D2Q9": 1, "D2Q37": 3, "D2Q17": 3}

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream; ``uniform()`` returns doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


def run(lattice, nx, ny, tau, sides=("periodic",) * 4, schemes=("cbc",) * 4,
        viscous="meso", dirichlet="eq", alpha_T=0.0, beta_P=0.0, t_inf=0.0,
        p_inf=None, inflow=None, rho0=1.0, storage="f64", steps=1, name="", alpha_V=0.0,
        u_ref=(0.0, 0.0)):
    """A run description understood by both the CUDA binding and the oracle
    (u_ref, the reference velocity of the CUDA path's stored populations, is
    a storage detail the oracle does not need)."""
    cs2 = CS2[lattice]
    return {
        "name": name, "lattice": lattice, "nx": int(nx), "ny": int(ny),
        "tau": float(tau), "rho0": float(rho0), "sides": list(sides),
        "schemes": list(schemes), "viscous": viscous,
        "dirichlet": dirichlet, "alpha_T": float(alpha_T), "beta_P": float(beta_P),
        "t_inf": float(t_inf), "alpha_V": float(alpha_V),
        "p_inf": list(p_inf) if p_inf is not None else [cs2 * rho0] * 4,
        "inflow": list(inflow) if inflow is not None else [rho0, 0.0, 0.0, 1.0],
        "storage": storage, "steps": int(steps), "u_ref": [float(u_ref[0]), float(u_ref[1])],
    }


# ---------------------------------------------------------------- fields ---

def grid(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx]
    return x.astype(np.float64), y.astype(np.float64)


def uniform(nx, ny, rho=1.0, ux=0.0, uy=0.0, T=1.0):
    shape = (ny, nx)
    return tuple(np.full(shape, float(v)) for v in (rho, ux, uy, T))


def gaussian_pulse(nx, ny, amp_rho, amp_T, width, center=None, rho0=1.0, T0=1.0,
                   u=(0.0, 0.0)):
    """rho = rho0 (1 + a_rho G), T = T0 (1 + a_T G), G = exp(-r^2 / (2 w^2))."""
    x, y = grid(nx, ny)
    cx, cy = center if center is not None else ((nx - 1) / 2.0, (ny - 1) / 2.0)
    G = np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * width * width))
    return (rho0 * (1.0 + amp_rho * G), np.full_like(G, u[0]), np.full_like(G, u[1]),
            T0 * (1.0 + amp_T * G))


def isentropic_vortex(nx, ny, lattice, Ma, strength=0.05, radius=20.0, center=None,
                      rho0=1.0, T0=1.0, gamma=2.0):
    """Isentropic vortex in a uniform stream U0 = Ma c_s along x.

    u = U0 e_x + eps (-(y-yc), x-xc)/R exp((1 - r^2/R^2)/2) with eps = strength U0
    (peak swirl eps at r = R); c_s^2 (T - T0) = -(gamma-1)/(2 gamma) eps^2
    exp(1 - r^2/R^2); rho = rho0 (T/T0)^(1/(gamma-1)).  gamma = c_p/c_v = 2
    in two dimensions (Sec. 2).
    """
    cs2 = CS2[lattice]
    U0 = Ma * math.sqrt(cs2)
    eps = strength * U0
    x, y = grid(nx, ny)
    xc, yc = center if center is not None else (nx / 4.0, (ny - 1) / 2.0)
    dx, dy = x - xc, y - yc
    r2 = (dx * dx + dy * dy) / (radius * radius)
    e = np.exp(0.5 * (1.0 - r2))
    ux = U0 - eps * dy / radius * e
    uy = eps * dx / radius * e
    T = T0 - (gamma - 1.0) / (2.0 * gamma) * eps * eps * np.exp(1.0 - r2) / cs2
    rho = rho0 * (T / T0) ** (1.0 / (gamma - 1.0))
    if lattice == "D2Q9":
        T = np.full_like(T, T0)
    return rho, ux, uy, T


def thermal_vortex(n, L, lattice, Ma=0.1, r=0.7, b=0.15, K=0.0, offset=0, isothermal=False):
    """The thermal vortex of the paper's Sec. 4.2 on an n x n grid whose
    window [offset, offset + L)^2 is the L x L benchmark domain: normalised
    coordinates x^ = 2 (x - 1) / (L - 1) - 1 (x counted from 1 in the
    window), a vortex at (K / (L - 1), 0) of radius r and strength b in a
    stream u0 = (Ma c_s, 0):  u = u0 + (5 c_s Ma / 2) 2^(-(x^2 + y^2) / b^2)
    (y, -x) and T = T0 + y^ (5 c_s Ma / 2) 2^(-(x^2 + y^2) / b^2) inside r
    (T = T0 for the iso-thermal vortex of Sec. 4.4), rho = rho0 = 1."""
    cs = math.sqrt(CS2[lattice])
    i = np.arange(n, dtype=np.float64) - offset
    xh = 2.0 * i / (L - 1) - 1.0
    X, Y = np.meshgrid(xh, xh)
    dx, dy = X - K / (L - 1), Y
    inside = dx * dx + dy * dy < r * r
    amp = 2.5 * cs * Ma * np.power(2.0, -(dx * dx + dy * dy) / (b * b))
    ux = Ma * cs + np.where(inside, amp * dy, 0.0)
    uy = np.where(inside, -amp * dx, 0.0)
    T = np.ones_like(X) if isothermal else 1.0 + np.where(inside, Y * amp, 0.0)
    return np.ones_like(X), ux, uy, T


def shear_wave(nx, ny, amp, k_axis="x", rho0=1.0):
    """u_y = A sin(2 pi x / nx) (k_axis "x") or u_x = A sin(2 pi y / ny)."""
    x, y = grid(nx, ny)
    rho, ux, uy, T = uniform(nx, ny, rho0)
    if k_axis == "x":
        uy = amp * np.sin(2.0 * np.pi * x / nx)
    else:
        ux = amp * np.sin(2.0 * np.pi * y / ny)
    return rho, ux, uy, T


def temperature_wave(nx, ny, amp, rho0=1.0):
    """T = 1 + A sin(2 pi x / nx) at uniform pressure (rho T = rho0), at rest."""
    x, _ = grid(nx, ny)
    T = 1.0 + amp * np.sin(2.0 * np.pi * x / nx)
    return rho0 / T, np.zeros_like(T), np.zeros_like(T), T


def smooth_random(nx, ny, seed, amp=1e-3, modes=3, lattice="D2Q37", u0=(0.0, 0.0)):
    """Sum of a few seeded periodic Fourier modes on each field (tests)."""
    rng = SplitMix64(seed)
    x, y = grid(nx, ny)
    out = []
    for f, base in enumerate((1.0, u0[0], u0[1], 1.0)):
        v = np.full((ny, nx), base)
        for _ in range(modes):
            kx = int(rng.uniform(0, 3))
            ky = int(rng.uniform(0, 3))
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-amp, amp)
            v = v + a * np.cos(2 * math.pi * (kx * x / nx + ky * y / ny) + ph)
        out.append(v)
    if lattice == "D2Q9":
        out[3] = np.ones((ny, nx))
    return tuple(out)


# ------------------------------------------------------------- workloads ---

def pulse_d2q9(n=64, steps=200, storage="f64", viscous="fd", tau=0.6):
    """D2Q9 isothermal BGK, density pulse a = 1e-3, w = 5, centred, CBC on all
    four sides; 64 x 64 and 200 steps at full size."""
    cfg = run("D2Q9", n, n, tau, sides=("cbc",) * 4, schemes=("cbc",) * 4,
              viscous=viscous, storage=storage, steps=steps,
              name="D2Q9 %dx%d Gaussian density pulse, CBC on 4 sides" % (n, n))
    return cfg, gaussian_pulse(n, n, 1e-3, 0.0, 5.0)


def pulse_d2q9_periodic_reference(n=256, steps=200):
    """The periodic reference run on which the 64 x 64 window is cropped."""
    cfg = run("D2Q9", n, n, 0.6, steps=steps, name="D2Q9 %dx%d periodic reference" % (n, n))
    return cfg, gaussian_pulse(n, n, 1e-3, 0.0, 5.0)


def pulse_d2q37(n=256, alpha_T=0.5, seed=0, steps=2000, storage="f32", tau=0.8,
                width=8.0, offset=10.0, beta_P=0.0):
    """D2Q37 fourth-order Hermite thermal lattice, combined rho/T Gaussian pulse
    (a = 1e-3, w = 8), centre offset by a seeded uniform +-10 cells per axis,
    CBC-RELAX on all four sides with transversal relaxation alpha_T."""
    rng = SplitMix64(seed)
    ox = rng.uniform(-offset, offset)
    oy = rng.uniform(-offset, offset)
    c = ((n - 1) / 2.0 + ox, (n - 1) / 2.0 + oy)
    cfg = run("D2Q37", n, n, tau, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
              alpha_T=alpha_T, beta_P=beta_P, storage=storage, steps=steps,
              name="D2Q37 %dx%d Gaussian rho+T pulse, CBC-RELAX alpha_T=%g" % (n, n, alpha_T))
    return cfg, gaussian_pulse(n, n, 1e-3, 1e-3, width, center=c)


def vortex_d2q37(nx=1024, ny=512, Ma=0.1, steps=20000, storage="f32", tau=0.8,
                 radius=20.0, reference=None):
    """D2Q37 isentropic vortex (strength 0.05 U0, R = 20) convected by a stream
    U0 = Ma c_s: inflow equilibrium on the left, periodic top/bottom,
    CBC-RELAX on the right with alpha_T = Ma, beta_P = 0 (the paper's outlet
    setting for its vortex benchmark).  With `reference` (default: for FP32
    and FP16 storage) the CUDA path holds its populations relative to the
    stream's equilibrium (u_ref = (U0, 0))."""
    cs2 = CS2["D2Q37"]
    U0 = Ma * math.sqrt(cs2)
    if reference is None:
        reference = storage != "f64"
    cfg = run("D2Q37", nx, ny, tau,
              sides=("inflow", "cbc", "periodic", "periodic"),
              schemes=("cbc_relax",) * 4, alpha_T=Ma, beta_P=0.0,
              inflow=(1.0, U0, 0.0, 1.0), storage=storage, steps=steps,
              u_ref=(U0, 0.0) if reference else (0.0, 0.0),
              name="D2Q37 %dx%d isentropic vortex Ma=%g, inflow|CBC, periodic y" % (nx, ny, Ma))
    return cfg, isentropic_vortex(nx, ny, "D2Q37", Ma, radius=radius)


def sweep_batch(n_runs=96, seed=4, steps=1000, storage="f32", lo=128, hi=512, viscous="meso"):
    """Batched coefficient sweep: n_runs independent runs, each a D2Q9 or
    D2Q37 run by a seeded coin, grid sides uniform in {lo..hi}, tau uniform
    in [0.55, 1.0], the transversal and pressure relaxation coefficients
    (alpha_T, beta_P) uniform in [0, 1], CBC-RELAX on all four sides, and a
    Gaussian pulse (a = 1e-3, width 8, centre offset by +-10 cells) drawn
    from a per-run seed.  Returns [(cfg, fields), ...].

    The viscous vector is the paper's mesoscopic one by default (all 96 runs
    stay finite over 1000 steps); "fd" and "off" are the alternatives."""
    rng = SplitMix64(seed)
    out = []
    for r in range(n_runs):
        lat = "D2Q37" if rng.uniform() < 0.5 else "D2Q9"
        nx = lo + int(rng.uniform() * (hi - lo + 1))
        ny = lo + int(rng.uniform() * (hi - lo + 1))
        tau = rng.uniform(0.55, 1.0)
        alpha_T, beta_P = rng.uniform(), rng.uniform()
        ox, oy = rng.uniform(-10.0, 10.0), rng.uniform(-10.0, 10.0)
        cfg = run(lat, nx, ny, tau, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
                  viscous=viscous, alpha_T=alpha_T, beta_P=beta_P, storage=storage,
                  steps=steps, name="sweep run %d: %s %dx%d" % (r, lat, nx, ny))
        amp_T = 1e-3 if lat == "D2Q37" else 0.0
        f = gaussian_pulse(nx, ny, 1e-3, amp_T, 8.0,
                           center=((nx - 1) / 2.0 + ox, (ny - 1) / 2.0 + oy))
        out.append((cfg, f))
    return out


def gradient_pulse(nx=512, ny=256, steps=1500, storage="f32", ref_scale=4, alpha_T=0.5, beta_P=0.5,
                   tau=0.8, width=8.0):
    """Relaxation-parameter gradient workload: D2Q37 nx x ny, a combined
    rho/T Gaussian pulse (a = 1e-3, width 8) at the centre, CBC-RELAX on
    four sides without the viscous vector, P_inf = c_s^2 rho0; and its
    reference, the same pulse at the centre of a periodic grid ref_scale
    times larger per axis.  Returns (cfg, fields, ref_cfg, ref_fields,
    (x0, y0)) with (x0, y0) the crop origin in the reference grid."""
    cfg = run("D2Q37", nx, ny, tau, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4, viscous="off",
              alpha_T=alpha_T, beta_P=beta_P, storage=storage, steps=steps,
              name="D2Q37 %dx%d rho+T pulse, CBC-RELAX, gradient workload" % (nx, ny))
    f = gaussian_pulse(nx, ny, 1e-3, 1e-3, width)
    rx, ry = nx * ref_scale, ny * ref_scale
    x0, y0 = (rx - nx) // 2, (ry - ny) // 2
    ref_cfg = run("D2Q37", rx, ry, tau, storage=storage, steps=steps,
                  name="D2Q37 %dx%d periodic reference" % (rx, ry))
    ref_f = gaussian_pulse(rx, ry, 1e-3, 1e-3, width, center=(x0 + (nx - 1) / 2.0, y0 + (ny - 1) / 2.0))
    return cfg, f, ref_cfg, ref_f, (x0, y0)
