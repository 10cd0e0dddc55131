"""Batched stepping of many independent runs (one band and one persistent
bulk launch per lattice and storage a step, replayed as CUDA graphs): every
run of a batch must come out bit-identical to the same run stepped alone, and
within the parity bars of the FP64 oracle."""

import numpy as np
import pytest

import lbm_workloads as W
import oracle

pytestmark = pytest.mark.gpu


def lbm():
    import paper_2307_16766_gb300 as m
    return m


def _mixed_runs():
    """Uneven sizes, every lattice, two storages, all side kinds, and runs
    whose relaxation times and characteristic parameters differ."""
    cs2_37, cs2_17 = W.CS2["D2Q37"], W.CS2["D2Q17"]
    runs = []
    cfg = W.run("D2Q9", 64, 48, 0.6, sides=("cbc",) * 4, schemes=("cbc",) * 4, viscous="fd")
    runs.append((dict(cfg, storage="f64"), W.gaussian_pulse(64, 48, 1e-3, 0.0, 5.0)))
    cfg = W.run("D2Q37", 96, 70, 0.8, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4,
                alpha_T=0.5, beta_P=0.3, p_inf=[cs2_37 * 1.0001] * 4)
    runs.append((dict(cfg, storage="f32"), W.gaussian_pulse(96, 70, 1e-3, 1e-3, 6.0, center=(40.2, 31.7))))
    cfg = W.run("D2Q37", 37, 130, 0.55, sides=("cbc", "cbc", "periodic", "periodic"),
                schemes=("lodi_relax",) * 4, viscous="meso", alpha_T=0.1, beta_P=0.9)
    runs.append((dict(cfg, storage="f32"), W.smooth_random(37, 130, seed=3, amp=1e-3, u0=(0.01, 0.0))))
    cfg = W.run("D2Q37", 150, 44, 1.0, sides=("inflow", "cbc", "periodic", "periodic"),
                schemes=("cbc_relax",) * 4, alpha_T=0.5, inflow=(1.0, 0.03, 0.0, 1.0))
    runs.append((dict(cfg, storage="f64"), W.smooth_random(150, 44, seed=5, amp=1e-3, u0=(0.03, 0.0))))
    cfg = W.run("D2Q37", 48, 40, 0.7)                       # periodic: no band tiles
    runs.append((dict(cfg, storage="f32"), W.smooth_random(48, 40, seed=7, amp=1e-3)))
    cfg = W.run("D2Q17", 41, 31, 0.75, sides=("cbc",) * 4, schemes=("cbc",) * 4, dirichlet="neep",
                alpha_T=0.3, beta_P=0.2, p_inf=[cs2_17 * 1.0002] * 4)
    runs.append((dict(cfg, storage="f32"), W.gaussian_pulse(41, 31, 1e-3, 1e-3, 3.5, center=(19.4, 14.1))))
    cfg = W.run("D2Q37", 9, 9, 0.9, sides=("cbc",) * 4, schemes=("cbc_relax",) * 4, alpha_T=0.5,
                viscous="fd")
    runs.append((dict(cfg, storage="f32"), W.gaussian_pulse(9, 9, 1e-3, 1e-3, 2.0)))
    cfg = W.run("D2Q37", 80, 60, 0.65, sides=("zg", "cbc", "periodic", "periodic"), schemes=("cbc_relax",) * 4,
                dirichlet="reg", viscous="off", alpha_T=1.0)
    runs.append((dict(cfg, storage="f32"), W.gaussian_pulse(80, 60, 1e-3, 1e-3, 5.0)))
    return runs


def _alone(cfg, fields, steps):
    sim = lbm().Simulation(cfg).init_fields(*fields)
    sim.step(steps)
    out = sim.macros()
    sim.close()
    return out


def _assert_bitwise(a, b, what):
    for name, x, y in zip(("rho", "ux", "uy", "T"), a, b):
        assert np.all(np.isfinite(x)), (what, name)
        assert np.array_equal(x, y), (what, name, np.abs(x - y).max())


def test_batch_runs_are_bit_identical_to_runs_stepped_alone(tmp_path, monkeypatch):
    monkeypatch.setenv("LBM_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    runs = _mixed_runs()
    B = lbm().Batch([c for c, _ in runs])
    for r, (_, f) in enumerate(runs):
        B[r].init_fields(*f)
    # eager steps while inflow buffers are filled, then graph replays of
    # both parities across several calls
    for n in (1, 2, 5, 3):
        B.step(n)
    assert all(B[r].steps_done == 11 for r in range(len(B)))
    for r, (c, f) in enumerate(runs):
        _assert_bitwise(B[r].macros(), _alone(c, f, 11), (r, c["lattice"], c["storage"]))
    B.close()


def test_batch_f64_runs_match_the_oracle():
    runs = [x for x in _mixed_runs() if x[0]["storage"] == "f64"]
    B = lbm().Batch([c for c, _ in runs])
    for r, (_, f) in enumerate(runs):
        B[r].init_fields(*f)
    B.step(40)
    for r, (c, f) in enumerate(runs):
        ref = oracle.Sim(c).init(*f).step(40).macros()
        got = B[r].macros()
        for x, y in zip(got, ref):
            assert np.abs(x - y).max() <= 1e-12 * max(1.0, np.abs(y).max()), r
    B.close()


def test_batch_of_many_uneven_runs():
    """A parameter-scan-like batch: 40 D2Q37 FP32 runs of uneven sizes,
    relaxation times and characteristic parameters, checked bit for bit
    against a sample of the runs stepped alone."""
    rng = np.random.default_rng(11)
    cfgs, fields = [], []
    for r in range(40):
        nx, ny = int(rng.integers(9, 120)), int(rng.integers(9, 120))
        # the mesoscopic viscous stencil needs 3 M + 3 = 12 nodes across
        cfg = W.run("D2Q37", nx, ny, float(rng.uniform(0.55, 1.0)), sides=("cbc",) * 4,
                    viscous="meso" if min(nx, ny) >= 12 else "fd",
                    schemes=("cbc_relax",) * 4, alpha_T=float(rng.uniform(0, 1)),
                    beta_P=float(rng.uniform(0, 1)))
        cfgs.append(dict(cfg, storage="f32"))
        fields.append(W.gaussian_pulse(nx, ny, 1e-3, 1e-3, max(2.0, min(nx, ny) / 8)))
    B = lbm().Batch(cfgs)
    for r in range(40):
        B[r].init_fields(*fields[r])
    B.step(25)
    for r in (0, 7, 19, 33, 39):
        _assert_bitwise(B[r].macros(), _alone(cfgs[r], fields[r], 25), r)
    B.close()


def test_autotune_result_is_cached_and_reused(tmp_path, monkeypatch):
    path = tmp_path / "cache" / "tune.txt"
    monkeypatch.setenv("LBM_AUTOTUNE_CACHE", str(path))
    runs = _mixed_runs()[1:3]
    B = lbm().Batch([c for c, _ in runs])
    assert B.ctas_per_sm("D2Q37", "f32") == 0
    for r, (_, f) in enumerate(runs):
        B[r].init_fields(*f)
    B.step(1)
    m = B.ctas_per_sm("D2Q37", "f32")
    assert 1 <= m <= 5
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].endswith(" %d" % m)
    B.close()
    # a planted entry is what the next batch of that bucket uses
    path.write_text(lines[0].rsplit(" ", 1)[0] + " 2\n")
    B = lbm().Batch([c for c, _ in runs])
    for r, (_, f) in enumerate(runs):
        B[r].init_fields(*f)
    B.step(2)
    assert B.ctas_per_sm("D2Q37", "f32") == 2
    assert len(path.read_text().splitlines()) == 1
    B.close()


def test_batch_rejects_runs_stepped_apart(monkeypatch):
    monkeypatch.setenv("LBM_AUTOTUNE_CACHE", "")
    m = lbm()
    runs = _mixed_runs()[1:3]
    B = m.Batch([c for c, _ in runs])
    with pytest.raises(m.LbmError):
        B.step(1)                      # runs not initialised
    for r, (_, f) in enumerate(runs):
        B[r].init_fields(*f)
    B.step(1)
    m.lbm_step(B[0].handle, 1)
    with pytest.raises(m.LbmError, match="apart"):
        B.step(1)
    B.close()
