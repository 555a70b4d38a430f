"""The seeded input generators (no evaluator arithmetic here)."""
import numpy as np

import blip_inputs as bi


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    # (x += 0x9E3779B97F4A7C15, then the finaliser).
    out = bi.raw_u64(np.uint64(0), np.arange(3, dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                     0x06C45D188009454F]


def test_uniform_and_normal_moments():
    k = bi.stream_key(1, 2)
    u = bi.uniform(k, np.arange(200000, dtype=np.uint64))
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    z = bi.normal(k, 0, 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2


def test_normal_ranges_are_cut_independent():
    k = bi.stream_key(9)
    full = bi.normal(k, 0, 101)
    assert np.array_equal(np.concatenate([bi.normal(k, 0, 37), bi.normal(k, 37, 64)]), full)


def test_table_is_deterministic_chunk_independent_and_normalised():
    a = bi.smooth_random_table((8, 9, 10), 5, seed=3, orb_chunk=2, threads=1)
    b = bi.smooth_random_table((8, 9, 10), 5, seed=3, orb_chunk=5, threads=4)
    assert np.array_equal(a, b)
    # orbital l does not depend on n_orb
    c = bi.smooth_random_table((8, 9, 10), 3, seed=3)
    assert np.array_equal(a[..., :3], c)
    rms = np.sqrt((a ** 2).mean(axis=(0, 1, 2)))
    assert np.allclose(rms, 1.0)
    # smooth: on a 24-point axis, sigma = 3 modes gives a lag-1 correlation
    # of about exp(-(2 pi / 24)^2 * 9 / 4) = 0.86
    s = bi.smooth_random_table((24, 24, 24), 2, seed=3)
    corr = (s * np.roll(s, 1, axis=2)).mean()
    assert 0.75 < corr < 0.95


def test_complex_table():
    a = bi.smooth_random_table((6, 6, 6), 2, seed=1, is_complex=True)
    assert a.dtype == np.complex128
    assert np.allclose(np.sqrt((np.abs(a) ** 2).mean(axis=(0, 1, 2))), 1.0)
    assert np.abs(a.imag).max() > 0.1


def test_walker_positions_and_offsets():
    lat = bi.tetragonal_lattice(17.4, 11.2)
    pos, offs = bi.walker_positions(lat, 4, 10, [1, 3, 0, 10], seed=5)
    assert offs.tolist() == [0, 1, 4, 4, 14] and pos.shape == (14, 3)
    sizes = bi.ragged_batch_sizes(1000, 1, 512, seed=2)
    assert sizes.min() >= 1 and sizes.max() <= 512 and 200 < sizes.mean() < 310


def test_named_workloads():
    w = bi.workload("cubic16")
    p, offs = w.positions()
    assert p.shape == (64, 3) and offs.tolist() == [0, 64]
    assert (p >= 0).all() and (p < 10.0).all()
    w = bi.workload("tio2_batch", batch=8)
    p, offs = w.positions()
    assert p.shape == (256 * 8, 3) and offs[-1] == 2048


def test_spectral_table_orbitals_are_independent_and_normalised():
    torch = __import__("pytest").importorskip("torch")
    a = bi.spectral_table((12, 10, 8), 5, seed=4, sigma=1.5, chunk=2)
    b = bi.spectral_table((12, 10, 8), range(3, 5), seed=4, sigma=1.5, chunk=1)
    assert a.shape == (12, 10, 8, 5) and a.dtype == torch.complex128
    assert torch.allclose(a[..., 3:5], b, rtol=0, atol=1e-13)
    rms = torch.sqrt((a.abs() ** 2).mean(dim=(0, 1, 2)))
    assert torch.allclose(rms, torch.ones(5, dtype=torch.float64))
    # smooth: lag-1 correlation along the 12-point axis is high
    c = (a * torch.roll(a, 1, dims=0).conj()).real.mean().item()
    assert c > 0.5


def test_spectral_table_matches_the_gaussian_filter_spectrum():
    """The power spectrum of the table falls off as exp(-|m|^2 / sigma^2)."""
    a = bi.spectral_table((24, 24, 24), 16, seed=9, sigma=3.0).numpy()
    f = np.fft.fftn(a, axes=(0, 1, 2))
    pw = (np.abs(f) ** 2).mean(axis=-1)
    m = np.fft.fftfreq(24) * 24
    r0 = pw[0, 0, 0]
    for k in (2, 4):
        expect = np.exp(-(k * k) / 9.0)
        got = np.mean([pw[k, 0, 0], pw[-k, 0, 0], pw[0, k, 0], pw[0, 0, k]]) / r0
        assert 0.3 * expect < got < 3.0 * expect
