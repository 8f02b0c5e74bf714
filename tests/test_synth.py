"""Seeded input generators: published SplitMix64 outputs, permutation and phantom invariants."""
import numpy as np

from paper_1605_00133_gb300 import presets, synth


def test_splitmix64_published_outputs():
    """Outputs of the SplitMix64 definition (Steele, Lea, Flood 2014) for seeds 0 and 1234567."""
    assert [int(v) for v in synth.splitmix64(0, 4)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(v) for v in synth.splitmix64(1234567, 3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_stream_is_counter_based():
    s = synth.Stream(42)
    a = s.raw(5)
    b = s.raw(3)
    assert np.array_equal(np.concatenate([a, b]), synth.splitmix64(42, 8))
    u = synth.Stream(42).uniform(1000)
    assert u.min() >= 0 and u.max() < 1


def test_fisher_yates_is_a_seeded_permutation():
    p = synth.fisher_yates(1000, 3)
    assert np.array_equal(np.sort(p), np.arange(1000))
    assert np.array_equal(p, synth.fisher_yates(1000, 3))
    assert not np.array_equal(p, synth.fisher_yates(1000, 4))


def test_index_sets():
    idx = synth.rsp_indices(16384, 2048, 0)
    assert idx.dtype == np.int32 and len(np.unique(idx)) == 2048 and np.all(np.diff(idx) > 0)
    perm, rows = synth.shd_pattern(16384, 2048, 0)
    assert np.array_equal(np.sort(perm), np.arange(16384))
    assert len(np.unique(rows)) == 2048 and rows.max() < 16384
    g = synth.gsp_indices(8, 8, 2)
    assert list(g[:4]) == [0, 2, 4, 6] and len(g) == 16


def test_phantoms():
    w = presets.workload("c1")
    p = w.p0()
    assert p.shape == (32, 32, 32) and p.max() > 0.4
    t = synth.branching_tubes((32, 48, 48), 5, 1, pml=4)
    assert t.min() >= 0 and t.max() <= 1 and t.max() > 0.05
    assert np.all(t[:4] == 0) and np.all(t[:, :, -4:] == 0)
    assert np.array_equal(t, synth.branching_tubes((32, 48, 48), 5, 1, pml=4))


def test_noise_level():
    f = np.ones((100, 100))
    n = synth.add_relative_noise(f, 0.01, 5) - f
    assert abs(n.std() - 0.01) < 1e-3


def test_band_limited_upsampling_keeps_the_coarse_values():
    from paper_1605_00133_gb300 import synth
    v = np.random.default_rng(3).standard_normal((8, 6, 10))
    b = synth.band_limit(v)
    assert np.abs(synth.band_limit(b) - b).max() < 1e-12
    u = synth.upsample2(b)
    assert u.shape == (16, 12, 20)
    assert np.abs(u[::2, ::2, ::2] - b).max() < 1e-12
    # the interpolant has no content above the coarse band
    U = np.fft.fftn(u)
    assert np.abs(U[4:12]).max() < 1e-9 * np.abs(U).max()
