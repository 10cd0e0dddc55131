"""The seeded input generators: reproducible and within the stated ranges."""
import numpy as np

import lbm_workloads as W


def test_splitmix64_matches_its_published_first_outputs():
    # SplitMix64 seeded with 0: the first outputs of the reference generator
    # (Steele, Lea & Flood 2014; also the seeding routine of xoshiro).
    r = W.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                0x06C45D188009454F]


def test_sweep_batch_is_seeded_and_in_range():
    a = W.sweep_batch(96)
    b = W.sweep_batch(96)
    assert len(a) == 96
    lats = set()
    for (ca, fa), (cb, fb) in zip(a, b):
        assert ca == cb
        for x, y in zip(fa, fb):
            assert np.array_equal(x, y)
        assert 128 <= ca["nx"] <= 512 and 128 <= ca["ny"] <= 512
        assert 0.55 <= ca["tau"] <= 1.0
        assert 0.0 <= ca["alpha_T"] <= 1.0 and 0.0 <= ca["beta_P"] <= 1.0
        assert ca["sides"] == ["cbc"] * 4 and ca["storage"] == "f32"
        assert fa[0].shape == (ca["ny"], ca["nx"])
        lats.add(ca["lattice"])
        if ca["lattice"] == "D2Q9":
            assert np.all(fa[3] == 1.0)           # isothermal lattice: no T pulse
    assert lats == {"D2Q9", "D2Q37"}
    sizes = {(c["nx"], c["ny"]) for c, _ in a}
    assert len(sizes) > 90                          # uneven
    assert W.sweep_batch(4, seed=5)[0][0] != a[0][0]


def test_gradient_pulse_reference_is_centred_on_the_crop():
    cfg, f, rcfg, rf, (x0, y0) = W.gradient_pulse(nx=64, ny=32, ref_scale=4)
    assert (rcfg["nx"], rcfg["ny"]) == (256, 128) and rcfg["sides"] == ["periodic"] * 4
    assert cfg["viscous"] == "off" and cfg["sides"] == ["cbc"] * 4
    for a, b in zip(f, rf):
        assert np.allclose(b[y0:y0 + 32, x0:x0 + 64], a, rtol=0.0, atol=1e-15)
