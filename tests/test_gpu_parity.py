"""Parity of the CUDA path with the FP64 CPU oracle, element by element.

Error measure per field (the reading of "relative" used throughout):
  rel_Z = max |Z_gpu - Z_ref| / max |Z_ref|,  Z in {rho, T};
  rel_u = max(|ux_gpu - ux_ref|, |uy_gpu - uy_ref|) / max(|ux_ref|, |uy_ref|).
Bars: FP64 storage 1e-12, FP32 storage 1e-5 after the stated step counts;
FP16 storage errors are reported per field against a loose bound.
"""
import functools

import numpy as np
import pytest

import lbm_workloads as W
import oracle

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def lbm():
    import paper_2307_16766_gb300 as m
    return m


def gpu_run(cfg, fields, steps):
    sim = lbm().Simulation(cfg).init_fields(*fields)
    sim.step(steps)
    out = sim.macros()
    sim.close()
    return out


@functools.lru_cache(maxsize=None)
def _oracle_cached(key):
    cfg, fields, steps = _ORACLE_ARGS[key]
    return oracle.Sim(cfg).init(*fields).step(steps).macros()


_ORACLE_ARGS = {}


def oracle_run(cfg, fields, steps, key=None):
    if key is None:
        return oracle.Sim(cfg).init(*fields).step(steps).macros()
    _ORACLE_ARGS[key] = (cfg, fields, steps)
    return _oracle_cached(key)


def rel_errors(got, ref):
    rho, ux, uy, T = got
    r_rho, r_ux, r_uy, r_T = ref
    umax = max(np.abs(r_ux).max(), np.abs(r_uy).max())
    return {
        "rho": np.abs(rho - r_rho).max() / np.abs(r_rho).max(),
        "u": max(np.abs(ux - r_ux).max(), np.abs(uy - r_uy).max()) / umax,
        "T": np.abs(T - r_T).max() / np.abs(r_T).max(),
    }


def assert_parity(cfg, fields, steps, storage="f64", key=None):
    c = dict(cfg)
    c["storage"] = storage
    got = gpu_run(c, fields, steps)
    ref = oracle_run(cfg, fields, steps, key)
    for a in got:
        assert np.all(np.isfinite(a))
    e = rel_errors(got, ref)
    tol = TOL[storage]
    assert max(e.values()) < tol, (storage, e)
    return e


# ------------------------------------------------------------ D2Q9 cases ---

def test_d2q9_pulse_64_full_200_steps():
    """64 x 64 D2Q9 density pulse, CBC on four sides (-FD viscous), 200 steps."""
    cfg, f = W.pulse_d2q9(64, 200)
    assert_parity(cfg, f, 200)


@pytest.mark.parametrize("scheme", ["lodi", "lodi_relax", "cbc", "cbc_relax"])
@pytest.mark.parametrize("vis,dirichlet", [("meso", "eq"), ("fd", "neep"), ("off", "eq")])
def test_d2q9_schemes(scheme, vis, dirichlet):
    n, m = 45, 38
    cfg = W.run("D2Q9", n, m, 0.65, sides=("cbc",) * 4, schemes=(scheme,) * 4, viscous=vis,
                dirichlet=dirichlet, alpha_T=0.4, beta_P=0.3, p_inf=[W.CS2["D2Q9"] * 1.0005] * 4)
    f = W.gaussian_pulse(n, m, 1e-3, 0.0, 4.0, center=(20.3, 17.6), u=(0.01, -0.02))
    assert_parity(cfg, f, 90)


@pytest.mark.parametrize("sides", [("zg",) * 4, ("inflow", "zg", "periodic", "periodic"),
                                   ("periodic",) * 4, ("cbc", "cbc", "periodic", "periodic")])
def test_d2q9_side_kinds(sides):
    n, m = 70, 33
    cfg = W.run("D2Q9", n, m, 0.7, sides=sides, schemes=("cbc_relax",) * 4, alpha_T=0.2,
                inflow=(1.0, 0.03, 0.0, 1.0))
    f = W.smooth_random(n, m, seed=5, amp=1e-3, lattice="D2Q9", u0=(0.02, 0.0))
    assert_parity(cfg, f, 120)


# ----------------------------------------------------------- D2Q37 cases ---

def test_d2q37_pulse_ragged_grid():
    """150 x 70 (two bulk tiles plus a ragged tail per row), CBC-RELAX with
    mesoscopic viscous terms on four sides, 120 steps."""
    cfg = W.run("D2Q37", 150, 70, 0.8, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
                alpha_T=0.5, beta_P=0.1)
    f = W.gaussian_pulse(150, 70, 1e-3, 1e-3, 6.0, center=(70.2, 33.9))
    assert_parity(cfg, f, 120)


@pytest.mark.parametrize("scheme", ["lodi", "lodi_relax", "cbc", "cbc_relax"])
@pytest.mark.parametrize("vis", ["meso", "fd", "off"])
@pytest.mark.parametrize("dirichlet", ["eq", "neep"])
def test_d2q37_schemes(scheme, vis, dirichlet):
    n, m = 37, 29
    cs2 = W.CS2["D2Q37"]
    cfg = W.run("D2Q37", n, m, 0.75, sides=("cbc",) * 4, schemes=(scheme,) * 4, viscous=vis,
                dirichlet=dirichlet, alpha_T=0.3, beta_P=0.2, p_inf=[cs2 * 1.0002] * 4)
    f = W.gaussian_pulse(n, m, 1e-3, 1e-3, 3.5, center=(17.4, 13.1), u=(0.01, 0.005))
    assert_parity(cfg, f, 60)


@pytest.mark.parametrize("lat,vis", [("D2Q37", "meso"), ("D2Q37", "fd"), ("D2Q17", "meso"), ("D2Q9", "fd")])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_viscous_relaxation_alpha_V(lat, vis, storage):
    """CBC-RELAX with the viscous term relaxed towards 0 at rate alpha_V = 0.6
    in the incoming amplitudes (an extension of Eq. CBC-Relax); a pulse that
    crosses two sides and a corner."""
    n, m = 41, 33
    cs2 = W.CS2[lat]
    cfg = W.run(lat, n, m, 0.75, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4, viscous=vis,
                alpha_T=0.3, beta_P=0.2, p_inf=[cs2 * 1.0002] * 4, alpha_V=0.6)
    f = W.gaussian_pulse(n, m, 1e-3, 1e-3 if lat != "D2Q9" else 0.0, 3.5, center=(9.4, 8.1),
                         u=(0.01, 0.005))
    assert_parity(cfg, f, 60, storage, "alpha_V_%s_%s" % (lat, vis))


@pytest.mark.parametrize("sides", [("zg",) * 4, ("inflow", "zg", "zg", "zg"),
                                   ("periodic",) * 4, ("periodic", "periodic", "cbc", "cbc")])
def test_d2q37_side_kinds(sides):
    n, m = 66, 40
    cfg = W.run("D2Q37", n, m, 0.8, sides=sides, schemes=("cbc_relax",) * 4, alpha_T=0.5,
                inflow=(1.0, 0.04, 0.0, 1.0))
    f = W.smooth_random(n, m, seed=9, amp=1e-3, u0=(0.01, 0.0))
    assert_parity(cfg, f, 100)


def test_d2q37_vortex_through_outlet_small():
    """Isentropic vortex convected through a CBC outlet (inflow left,
    periodic y) on a reduced grid, Ma = 0.3, 400 steps."""
    cfg, f = W.vortex_d2q37(160, 48, Ma=0.3, steps=400, storage="f64", radius=8.0)
    assert_parity(cfg, f, 400)


@pytest.mark.parametrize("n,vis", [(9, "fd"), (12, "meso")])
def test_d2q37_minimal_grid(n, vis):
    """Smallest admissible grids: 2M + 3 = 9 nodes per open axis, 3M + 3 =
    12 with the mesoscopic viscous stencil (it reaches M + 2 nodes below
    x_f)."""
    cfg = W.run("D2Q37", n, n, 0.9, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4, alpha_T=0.5,
                viscous=vis)
    f = W.gaussian_pulse(n, n, 1e-3, 1e-3, 2.0)
    assert_parity(cfg, f, 50)


# ----------------------------------------------------------- D2Q17 cases ---

@pytest.mark.parametrize("scheme", ["lodi", "lodi_relax", "cbc", "cbc_relax"])
@pytest.mark.parametrize("vis,dirichlet", [("meso", "eq"), ("fd", "neep"), ("off", "eq")])
def test_d2q17_schemes(scheme, vis, dirichlet):
    """D2Q17 (Tab. d2q17, Eq. feq-3) with every scheme on four CBC sides."""
    n, m = 41, 31
    cs2 = W.CS2["D2Q17"]
    cfg = W.run("D2Q17", n, m, 0.75, sides=("cbc",) * 4, schemes=(scheme,) * 4, viscous=vis,
                dirichlet=dirichlet, alpha_T=0.3, beta_P=0.2, p_inf=[cs2 * 1.0002] * 4)
    f = W.gaussian_pulse(n, m, 1e-3, 1e-3, 3.5, center=(19.4, 14.1), u=(0.01, 0.005))
    assert_parity(cfg, f, 60)


@pytest.mark.parametrize("sides", [("zg",) * 4, ("inflow", "cbc", "periodic", "periodic"),
                                   ("periodic",) * 4, ("periodic", "periodic", "cbc", "cbc")])
def test_d2q17_side_kinds(sides):
    n, m = 150, 44
    cfg = W.run("D2Q17", n, m, 0.8, sides=sides, schemes=("cbc_relax",) * 4, alpha_T=0.5,
                inflow=(1.0, 0.03, 0.0, 1.0))
    f = W.smooth_random(n, m, seed=13, amp=1e-3, lattice="D2Q17", u0=(0.01, 0.0))
    assert_parity(cfg, f, 100)


def test_d2q17_f32_and_f16_storage(capsys):
    """FP32 storage within 1e-5 of the FP64 oracle; FP16 reported per field.
    The FP16 run leaves out the viscous vector: half-precision rounding noise
    (~1e-7) seeds the growth of the viscous terms at a boundary at rest (a
    property of the method, see the stability findings), which reaches 5e-3
    on rho after 300 steps on D2Q17 with the mesoscopic form."""
    cfg = W.run("D2Q17", 128, 96, 0.8, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
                alpha_T=1.0, beta_P=0.0)
    f = W.gaussian_pulse(128, 96, 1e-3, 1e-3, 6.0, center=(60.3, 50.2))
    assert_parity(cfg, f, 300, storage="f32")
    cfg = dict(cfg, viscous="off")
    c = dict(cfg)
    c["storage"] = "f16"
    e = rel_errors(gpu_run(c, f, 300), oracle_run(cfg, f, 300))
    with capsys.disabled():
        print("\nFP16 storage, D2Q17 128x96, 300 steps: rel errors", {k: "%.2e" % v for k, v in e.items()})
    assert e["rho"] < 1e-5 and e["T"] < 1e-5 and e["u"] < 1e-1


# ---------------------------------------- regularised Dirichlet condition ---

@pytest.mark.parametrize("lat", ["D2Q9", "D2Q17", "D2Q37"])
@pytest.mark.parametrize("vis", ["meso", "off"])
def test_regularised_dirichlet(lat, vis):
    """NEEP with the non-equilibrium part of x_f projected onto the Hermite
    polynomials of orders 2 (and 3 on the thermal lattices)."""
    n, m = 44, 36
    cs2 = W.CS2[lat]
    cfg = W.run(lat, n, m, 0.75, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4, viscous=vis,
                dirichlet="reg", alpha_T=0.5, beta_P=0.2, p_inf=[cs2 * 1.0002] * 4)
    f = W.gaussian_pulse(n, m, 1e-3, 1e-3 if lat != "D2Q9" else 0.0, 3.5, center=(20.4, 16.1),
                         u=(0.01, 0.005))
    assert_parity(cfg, f, 80)


def test_regularised_dirichlet_f32():
    """FP32 storage within 1e-5.  The viscous vector is left out: with it, the
    storage rounding noise it amplifies at a boundary at rest (see the FP16
    cases) reaches 1.2e-5 of max|u| here; the FP64 cases above cover the
    regularised write with the mesoscopic vector."""
    cfg = W.run("D2Q37", 96, 64, 0.8, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
                dirichlet="reg", alpha_T=1.0, viscous="off")
    f = W.gaussian_pulse(96, 64, 1e-3, 1e-3, 5.0)
    assert_parity(cfg, f, 200, storage="f32")


# -------------------------------------------------- full-size workloads ---

@pytest.mark.parametrize("alpha", [0.5, 1.0])
def test_d2q37_pulse_256_full_2000_steps_f64(alpha):
    """D2Q37 256 x 256 rho+T pulse, CBC-RELAX on four sides, 2000 steps, FP64
    storage: 1e-12 of the oracle."""
    cfg, f = W.pulse_d2q37(256, alpha_T=alpha, steps=2000, storage="f64")
    cfg["viscous"] = "off"
    assert_parity(cfg, f, 2000, "f64", ("pulse256", alpha, 2000))


def _conditioning(cfg, f, steps):
    """The oracle's end state, max |u| over its run, and the FP64 GPU run
    from fields perturbed by 1e-10 (seeded) against it."""
    o = oracle.Sim(cfg).init(*f)
    umax_run = 0.0
    for _ in range(steps // 50):
        o.step(50)
        m = o.macros()
        umax_run = max(umax_run, np.abs(m[1]).max(), np.abs(m[2]).max())
    ref = o.macros()
    rng = np.random.default_rng(5)
    fp = tuple(a * (1.0 + 1e-10 * rng.standard_normal(a.shape)) if i in (0, 3) else a
               for i, a in enumerate(f))
    return ref, umax_run, rel_errors(gpu_run(cfg, fp, steps), ref)


def test_d2q37_pulse_256_full_2000_steps_f32_continuous_scheme(capsys):
    """alpha_T = 1 (the incoming-wave treatment continuous at Lambda = u_n =
    0), FP32 storage, 2000 steps.  By then the pulse has left and max |u| has
    fallen to ~5e-3 of its peak, so rel_u of the end state measures the
    problem's conditioning: the FP64 run from fields perturbed by 1e-10 lies
    1.4e-3 from the oracle there.  FP32 is held to 1e-5 in rho and T, to
    1e-5 of max |u| over the run in u (measured 4.9e-8), and its end-state
    rel_u (measured ~1e-5) below the conditioning figure; both are printed."""
    cfg, f = W.pulse_d2q37(256, alpha_T=1.0, steps=2000, storage="f64")
    cfg["viscous"] = "off"
    assert_parity(cfg, f, 150, "f32", ("pulse256", 1.0, 150))
    ref, umax_run, econd = _conditioning(cfg, f, 2000)
    got32 = gpu_run(dict(cfg, storage="f32"), f, 2000)
    e32 = rel_errors(got32, ref)
    du32 = max(np.abs(got32[1] - ref[1]).max(), np.abs(got32[2] - ref[2]).max())
    with capsys.disabled():
        print("\nalpha_T = 1, 2000 steps: FP32 rel errors", {k: "%.2e" % v for k, v in e32.items()},
              "| FP64 with 1e-10 perturbed fields", {k: "%.2e" % v for k, v in econd.items()},
              "| FP32 |du| / max|u| over the run %.2e" % (du32 / umax_run))
    assert e32["rho"] < 1e-5 and e32["T"] < 1e-5, e32
    assert du32 / umax_run < 1e-5, du32 / umax_run
    assert e32["u"] < econd["u"], (e32, econd)


def test_d2q37_pulse_256_f32_switching_scheme(capsys):
    """alpha_T = 0.5: the incoming-wave treatment of the waves with
    Lambda = u_n jumps by (1 - alpha_T) T_i when u_n changes sign (Sec. 3.2
    classifies by the sign of Lambda), and once the pulse has left, the
    boundary is nearly at rest and that switch amplifies any perturbation.
    FP32 storage meets 1e-5 while the pulse crosses the boundary (150 steps).
    After 2000 steps it does not (rel_u ~0.17 against the tiny residual
    flow); the FP64 run itself, with its initial fields perturbed by 1e-10
    (seeded), moves as far from the unperturbed FP64 oracle.  The test
    reports both and holds FP32 to within a factor of 3 of that conditioning
    figure, and reports the error against max |u| over the whole run."""
    cfg, f = W.pulse_d2q37(256, alpha_T=0.5, steps=2000, storage="f64")
    cfg["viscous"] = "off"
    assert_parity(cfg, f, 150, "f32", ("pulse256", 0.5, 150))
    ref, umax_run, econd = _conditioning(cfg, f, 2000)
    got32 = gpu_run(dict(cfg, storage="f32"), f, 2000)
    e32 = rel_errors(got32, ref)
    du32 = max(np.abs(got32[1] - ref[1]).max(), np.abs(got32[2] - ref[2]).max())
    with capsys.disabled():
        print("\nalpha_T = 0.5, 2000 steps: FP32 rel errors", {k: "%.2e" % v for k, v in e32.items()},
              "| FP64 with 1e-10 perturbed fields", {k: "%.2e" % v for k, v in econd.items()},
              "| FP32 |du| / max|u| over the run %.2e" % (du32 / umax_run))
    assert e32["rho"] < 1e-5 and e32["T"] < 1e-5, e32
    assert e32["u"] < 3.0 * econd["u"], (e32, econd)


def test_d2q37_pulse_256_meso_viscous_prefix():
    """The same workload with mesoscopic viscous terms and alpha_T = 0 over
    the first 300 steps (the scheme grows from a boundary at rest later)."""
    cfg, f = W.pulse_d2q37(256, alpha_T=0.0, steps=300, storage="f64")
    assert_parity(cfg, f, 300)


def test_d2q37_vortex_1024x512_full_grid_short():
    """The benchmark grid (1024 x 512 vortex, inflow | CBC, periodic y) in the
    launch configuration the benchmark times, checked on every node after 20
    steps in FP64 and FP32."""
    cfg, f = W.vortex_d2q37(1024, 512, Ma=0.1, steps=20, storage="f64")
    assert_parity(cfg, f, 20, "f64", "vortex1024")
    assert_parity(cfg, f, 20, "f32", "vortex1024")


@pytest.mark.parametrize("n,storage", [(4096, "f64"), (4096, "f32"), (7616, "f32")])
def test_d2q37_pulse_large_grid_window_matches_periodic_oracle(n, storage):
    """The 4096^2 throughput grid, and the largest D2Q37 grid the library
    accepts (7616^2: 37 x 7616^2 population values, just under 2^31, so the
    32-bit element offsets reach their limit), with the 256^2 pulse recipe
    (CBC-RELAX on four sides) in the launch configuration the benchmark
    times.  After 30 steps the disturbance has travelled ~35 cells and the
    stencils reach at most 90: the 256^2 window around the pulse must equal
    the oracle's 256^2 periodic run of the same pulse (the fields outside
    the window differ from the periodic images by the Gaussian tail at 128
    cells, e^-128), and the boundary layers, which the disturbance has not
    reached, must still hold the uniform state."""
    w, steps = 256, 30
    x0 = n // 2 - w // 2
    cfg, f = W.pulse_d2q37(n, storage=storage, steps=steps)
    rng = W.SplitMix64(0)                       # the recipe's centre offset
    ox, oy = rng.uniform(-10.0, 10.0), rng.uniform(-10.0, 10.0)
    centre = ((n - 1) / 2.0 + ox - x0, (n - 1) / 2.0 + oy - x0)
    got = gpu_run(cfg, f, steps)
    del f
    win = [a[x0:x0 + w, x0:x0 + w] for a in got]
    rcfg = W.run("D2Q37", w, w, cfg["tau"], storage="f64", steps=steps)
    ref = oracle_run(rcfg, W.gaussian_pulse(w, w, 1e-3, 1e-3, 8.0, center=centre), steps,
                     key="pulse_window_%d" % n)
    e = rel_errors(win, ref)
    assert max(e.values()) < TOL[storage], (n, storage, e)
    rho, ux, uy, T = got
    band = np.ones_like(rho, dtype=bool)
    band[3:-3, 3:-3] = False
    assert np.abs(rho[band] - 1.0).max() < 1e-6 and np.abs(T[band] - 1.0).max() < 1e-6
    assert max(np.abs(ux[band]).max(), np.abs(uy[band]).max()) < 1e-6


def test_d2q37_many_tiles_pulse_through_a_corner():
    """400 x 300 with four CBC-RELAX sides: 42 band tiles, more four-CTA
    clusters than fit on a GB300 at one per four SMs, so the band launch
    runs in more than one wave; the pulse crosses the W and S sides and the
    corner between them."""
    cs2 = W.CS2["D2Q37"]
    cfg = W.run("D2Q37", 400, 300, 0.8, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
                alpha_T=0.5, beta_P=0.3, p_inf=[cs2 * 1.0001] * 4, steps=80)
    f = W.gaussian_pulse(400, 300, 1e-3, 1e-3, 5.0, center=(24.3, 31.7))
    assert_parity(cfg, f, 80, "f64", "many_tiles")
    assert_parity(cfg, f, 80, "f32", "many_tiles")


@pytest.mark.parametrize("Ma", [0.1, 0.3])
def test_vortex_1024x512_20000_steps_fp32_fp16_against_fp64(Ma, capsys):
    """The benchmark grid's vortex (inflow | CBC-RELAX with the mesoscopic
    viscous vector, periodic y) at Ma = 0.1 and 0.3 over 20000 steps, FP32
    and FP16 storage (populations held relative to the stream's
    equilibrium, u_ref = (U0, 0)) against the FP64 path (which matches the
    oracle to 1e-12 over the first 2000 steps, below), per field.  FP32:
    every field within the 1e-5 target (with the plain shift u missed it:
    2.9e-5 and 4.2e-5, the rounding of populations of the stream's size).
    FP16: reported, with loose bars."""
    steps = 20000

    def run(storage):
        cfg, f = W.vortex_d2q37(1024, 512, Ma=Ma, steps=steps, storage=storage)
        return gpu_run(cfg, f, steps)

    ref = run("f64")
    res = {st: rel_errors(run(st), ref) for st in ("f32", "f16")}
    with capsys.disabled():
        print("\nvortex 1024x512 Ma=%.1f, %d steps, mesoscopic V, rel. errors vs FP64 (target 1e-5):" % (Ma, steps),
              {st: {k: "%.2e" % v for k, v in e.items()} for st, e in res.items()})
    assert max(res["f32"].values()) < 1e-5, res
    assert res["f16"]["rho"] < 5e-3 and res["f16"]["T"] < 5e-3 and res["f16"]["u"] < 2e-2, res


def test_d2q37_vortex_1024x512_2000_steps_f64_oracle():
    """The benchmark configuration (mesoscopic viscous vector) over 2000
    steps, FP64 storage, every node against the oracle (about a minute of
    oracle time on the host)."""
    cfg, f = W.vortex_d2q37(1024, 512, Ma=0.1, steps=2000, storage="f64")
    assert_parity(cfg, f, 2000, "f64", "vortex1024_2000")


def test_d2q37_vortex_1024x512_first_500_steps_f64():
    """The benchmark configuration as timed (mesoscopic viscous vector) over
    its first 500 steps, FP64 storage, every node against the oracle."""
    cfg, f = W.vortex_d2q37(1024, 512, Ma=0.1, steps=500, storage="f64")
    assert_parity(cfg, f, 500, "f64", "vortex1024_500")


def test_f16_storage_error_per_field(capsys):
    """FP16 storage (g / w in half precision, FP32 arithmetic): errors against
    the oracle are reported per field; they stay at the half-precision level."""
    cfg = W.run("D2Q37", 128, 96, 0.8, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
                alpha_T=0.5, viscous="off")
    f = W.gaussian_pulse(128, 96, 1e-3, 1e-3, 6.0)
    c = dict(cfg)
    c["storage"] = "f16"
    got = gpu_run(c, f, 300)
    ref = oracle_run(cfg, f, 300)
    e = rel_errors(got, ref)
    with capsys.disabled():
        print("\nFP16 storage, D2Q37 128x96, 300 steps: rel errors", {k: "%.2e" % v for k, v in e.items()})
    assert e["rho"] < 1e-5 and e["T"] < 1e-5 and e["u"] < 1e-1


# ---------------------------------------------------------- API behaviour ---

def test_bounded_tma_wait_gives_up_with_a_timeout_status():
    """With a wait limit of 0 the bulk kernel's first wait for its tensor
    copies runs out: the kernel records it, waits (bounded, 1 s) for the
    copies in flight and leaves; the macros call reports LBM_ERR_TIMEOUT and
    the context stays usable -- with the default limit restored, the same
    run matches the oracle again."""
    L = lbm()
    cfg, f = W.pulse_d2q37(64, alpha_T=0.5, steps=5, storage="f32", width=5.0, offset=3.0)
    sim = L.Simulation(cfg).init_fields(*f)
    L.lbm_set_wait_limit(sim.handle, 0.0)
    sim.step(2)
    with pytest.raises(L.LbmError) as e:
        sim.macros()
    assert e.value.code == -6
    L.lbm_set_wait_limit(sim.handle, 1.0)
    sim.init_fields(*f)
    sim.step(5)
    got = sim.macros()
    sim.close()
    e2 = rel_errors(got, oracle_run(dict(cfg, storage="f64"), f, 5))
    assert max(e2.values()) < 1e-5, e2


def test_saved_state_holds_no_leftover_workspace_bytes():
    """A handle's population buffers are zeroed at creation, so a saved
    state does not depend on what the workspace held before (the row
    padding x >= nx is never written by a kernel): two handles made on
    workspaces left dirty with different bytes save equal states."""
    import torch
    cfg = W.run("D2Q17", 200, 100, 0.8, sides=("cbc",) * 4, schemes=("cbc",) * 4,
                dirichlet="neep", storage="f32")
    f = W.gaussian_pulse(200, 100, 1e-3, 1e-3, 4.0)
    states = []
    for fill in (float("nan"), 7.0):
        junk = torch.full((64 << 20,), fill, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        del junk                         # back to the caching allocator, dirty
        sim = lbm().Simulation(cfg).init_fields(*f)
        sim.step(5)
        states.append(sim.get_state())
        sim.close()
    assert states[0] == states[1]


def test_checkpoint_resume_is_bit_exact():
    cfg, f = W.pulse_d2q37(64, alpha_T=0.5, steps=100, storage="f32", width=5.0, offset=3.0)
    sim = lbm().Simulation(cfg).init_fields(*f)
    sim.step(40)
    state = sim.get_state()
    sim.step(35)
    a = sim.macros()
    sim.set_state(state)
    assert sim.steps_done == 40
    sim.step(35)
    b = sim.macros()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    sim.close()


def test_zero_steps_and_device_fields():
    import torch
    cfg, f = W.pulse_d2q37(48, alpha_T=0.5, steps=0, storage="f64", width=4.0, offset=2.0)
    sim = lbm().Simulation(cfg).init_fields(*f)
    sim.step(0)
    got = sim.macros()
    for g, r in zip(got, f):
        assert np.abs(g - r).max() < 1e-15
    dev = [torch.tensor(a, device="cuda") for a in f]
    sim.init_fields(*dev)
    sim.step(10)
    a = sim.macros(device=True)
    sim.init_fields(*f)
    sim.step(10)
    b = sim.macros()
    for x, y in zip(a, b):
        assert np.array_equal(x.cpu().numpy(), y)
    sim.close()


def test_non_finite_fields_are_reported():
    m = lbm()
    cfg = W.run("D2Q9", 16, 16, 0.7)
    f = list(W.uniform(16, 16))
    f[0] = f[0].copy()
    f[0][3, 4] = np.nan
    sim = m.Simulation(cfg).init_fields(*f)
    sim.step(2)
    with pytest.raises(m.LbmError) as e:
        sim.macros()
    assert e.value.code == -4
    sim.close()


def test_phase_order_is_enforced():
    m = lbm()
    cfg = W.run("D2Q9", 16, 16, 0.7)
    sim = m.Simulation(cfg)
    with pytest.raises(m.LbmError) as e:
        sim.step(1)
    assert e.value.code == -5
    sim.init_fields(*W.uniform(16, 16))
    with pytest.raises(m.LbmError):
        sim.step_phase(1)
    sim.step_phase(0)
    with pytest.raises(m.LbmError):
        sim.macros()
    sim.step_phase(1)
    assert sim.steps_done == 1
    sim.close()


# ------------------------------------------- overlapped step schedule ---

def _phased(cfg, fields, steps):
    sim = lbm().Simulation(cfg).init_fields(*fields)
    for _ in range(steps):
        sim.step_phase(0)
        sim.step_phase(1)
    state = sim.get_state()
    sim.close()
    return state


def _overlapped(cfg, fields, steps, chunks=(1, 4)):
    sim = lbm().Simulation(cfg).init_fields(*fields)
    done, k = 0, 0
    while done < steps:
        n = min(chunks[k % len(chunks)], steps - done)
        sim.step(n)
        done += n
        k += 1
    state = sim.get_state()
    sim.close()
    return state


@pytest.mark.parametrize("case", [
    "vortex_inflow_cbc_periodic_y", "d2q37_four_cbc_f32", "d2q37_cbc_y_periodic_x_f16",
    "d2q9_four_cbc_f64", "d2q37_zg_x_periodic_y", "d2q37_interior_empty",
    "d2q37_fully_periodic", "d2q17_four_cbc_neep_f32"])
def test_overlapped_step_is_bit_identical_to_phased_step(case):
    """lbm_step runs the band kernel beside the bulk kernel on two streams;
    populations, strips and boundary state must equal those of the
    sequential phase 0 / phase 1 order bit for bit."""
    if case == "vortex_inflow_cbc_periodic_y":
        cfg, f = W.vortex_d2q37(160, 48, Ma=0.3, steps=60, storage="f32", radius=8.0)
    elif case == "d2q37_four_cbc_f32":
        cfg, f = W.pulse_d2q37(70, alpha_T=0.5, steps=60, storage="f32", width=5.0, offset=3.0)
    elif case == "d2q37_cbc_y_periodic_x_f16":
        cfg = W.run("D2Q37", 64, 40, 0.8, sides=("periodic", "periodic", "cbc", "cbc"),
                    schemes=("cbc_relax",) * 4, alpha_T=0.5, storage="f16")
        f = W.gaussian_pulse(64, 40, 1e-3, 1e-3, 4.0)
    elif case == "d2q9_four_cbc_f64":
        cfg, f = W.pulse_d2q9(48, steps=60)
    elif case == "d2q37_zg_x_periodic_y":
        cfg = W.run("D2Q37", 50, 30, 0.8, sides=("zg", "zg", "periodic", "periodic"), storage="f32")
        f = W.gaussian_pulse(50, 30, 1e-3, 1e-3, 4.0)
    elif case == "d2q37_interior_empty":
        cfg = W.run("D2Q37", 11, 12, 0.9, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
                    alpha_T=0.5, storage="f64", viscous="fd")
        f = W.gaussian_pulse(11, 12, 1e-3, 1e-3, 2.0)
    elif case == "d2q17_four_cbc_neep_f32":
        cfg = W.run("D2Q17", 48, 40, 0.8, sides=("cbc",) * 4, schemes=("cbc",) * 4,
                    dirichlet="neep", storage="f32")
        f = W.gaussian_pulse(48, 40, 1e-3, 1e-3, 4.0)
    else:
        cfg = W.run("D2Q37", 40, 24, 0.8, storage="f32")
        f = W.gaussian_pulse(40, 24, 1e-3, 1e-3, 4.0)
    a = _phased(cfg, f, 23)
    b = _overlapped(cfg, f, 23)
    assert a == b


def test_kernel_events_time_the_interior_launch():
    import torch
    m = lbm()
    cfg, f = W.vortex_d2q37(256, 64, Ma=0.1, steps=10, storage="f32", radius=8.0)
    sim = m.Simulation(cfg).init_fields(*f)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    for e in ev:
        e.record(sim.stream)       # creates the events
    m.lbm_set_kernel_events(sim.handle, [e.cuda_event for e in ev])
    sim.step(1)
    torch.cuda.synchronize()
    bulk, band = ev[0].elapsed_time(ev[1]), ev[3].elapsed_time(ev[4])
    assert 0.0 < bulk < 50.0 and 0.0 < band < 50.0
    assert ev[2].elapsed_time(ev[0]) >= 0.0 and ev[2].elapsed_time(ev[3]) >= 0.0
    sim.step_phase(0)
    sim.step_phase(1)              # phased: all five on the solver's stream, in order
    torch.cuda.synchronize()
    # order on one stream: step start (2), bulk (0, 1), band (3, 4)
    assert ev[2].elapsed_time(ev[0]) >= 0.0 and ev[0].elapsed_time(ev[1]) > 0.0
    assert ev[1].elapsed_time(ev[3]) >= 0.0 and ev[3].elapsed_time(ev[4]) > 0.0
    m.lbm_set_kernel_events(sim.handle, [])
    with pytest.raises(m.LbmError):
        m.lbm_set_kernel_events(sim.handle, [ev[0].cuda_event])
    sim.step(2)
    sim.close()


def test_step_replays_under_cuda_graph_capture():
    """The fork/join of lbm_step is capturable: a graph of two steps,
    replayed, reproduces eager stepping bit for bit."""
    import torch
    m = lbm()
    cfg, f = W.vortex_d2q37(160, 48, Ma=0.3, steps=30, storage="f32", radius=8.0)
    ref = m.Simulation(cfg).init_fields(*f)
    ref.step(2 + 2 * 5)
    want = ref.macros()
    ref.close()

    sim = m.Simulation(cfg).init_fields(*f)
    sim.step(2)                    # both buffers get their inflow nodes eagerly
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        m.lbm_set_stream(sim.handle, s.cuda_stream)
        m.lbm_step(sim.handle, 2)  # recorded only: the buffers do not advance
    for _ in range(5):
        g.replay()
    torch.cuda.synchronize()
    m.lbm_set_stream(sim.handle, torch.cuda.current_stream().cuda_stream)
    got = sim.macros()             # host counter: 4 steps, parity matches 12
    sim.close()
    for x, y in zip(want, got):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("storage,dirichlet", [("f32", "eq"), ("f16", "neep"), ("f32", "reg")])
def test_band_launch_width_does_not_change_results(storage, dirichlet):
    """With FP32 / FP16 storage each band CTA takes every band_ctas-th tile
    in turn (shared memory reused from tile to tile); one CTA for all tiles,
    three, and one per tile give the same bits.  A 160x128 pulse on four
    characteristic sides (corners included; over a dozen tiles) with the
    mesoscopic viscous vector."""
    cfg, f = W.pulse_d2q37(160, storage=storage)
    cfg = dict(cfg, ny=128, dirichlet=dirichlet)
    f = tuple(a[:128, :] for a in f)
    res = [gpu_run(dict(cfg, band_ctas=k), f, 40) for k in (0, 1, 3)]
    for other in res[1:]:
        for x, y in zip(res[0], other):
            assert np.array_equal(x, y)
    assert all(np.isfinite(a).all() for a in res[0])
