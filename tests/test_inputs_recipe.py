"""The seeded workloads hold the recipes the benchmark and the tests state for them
(sizes, wavenumber ranges, source statistics, arrival process), checked on the CPU from
the generated arrays alone.  The generators draw random numbers only; none of the
solver's arithmetic is involved."""
import numpy as np
import pytest

from paper_1012_5379_gb300 import inputs as I


def test_point_source_is_one_unit_at_the_centre():
    for dim, n in ((2, 127), (3, 15)):
        b = I.point_source(dim, n)
        assert b.shape == (n,) * dim and b.dtype == np.complex128
        assert np.count_nonzero(b) == 1 and b[((n - 1) // 2,) * dim] == 1.0


def test_random_source_is_unit_variance_complex_normal_and_seeded():
    b = I.random_source(2, 511, 7)
    assert b.shape == (511, 511) and b.dtype == np.complex128
    # E|b|^2 = 1, real and imaginary parts each of variance 1/2, mean 0 (261k samples)
    assert abs(np.mean(np.abs(b) ** 2) - 1.0) < 0.01
    assert abs(np.var(b.real) - 0.5) < 0.01 and abs(np.var(b.imag) - 0.5) < 0.01
    assert abs(np.mean(b)) < 0.01
    assert np.array_equal(b, I.random_source(2, 511, 7))
    assert not np.array_equal(b, I.random_source(2, 511, 8))


def test_bump_field_wavenumber_range_and_shape():
    """k(x) = 80 (1 + 0.3 g) with g clipped to [-1, 1]: k stays in [56, 104], varies
    smoothly (8 bumps of width 0.1), and is reproducible from its seed."""
    n = 63
    phi = I.bump_field(n, 1002)
    assert phi.shape == (n, n, n) and phi.dtype == np.float32
    k = np.sqrt(phi.astype(np.float64))
    g = k / 80.0 - 1.0
    assert g.min() >= -0.3 * (1 + 1e-6) and g.max() <= 0.3 * (1 + 1e-6)
    assert g.max() - g.min() > 0.1            # the bumps are there
    # neighbouring nodes (h = 1/64) differ by far less than the field's range
    assert np.max(np.abs(np.diff(k, axis=2))) < 0.25 * (k.max() - k.min())
    assert np.array_equal(phi, I.bump_field(n, 1002))


def test_cube_and_2d_workloads_match_their_configs():
    c = I.cube_3d(31)
    assert (c.dim, c.n, c.restart, c.tol, c.precision) == (3, 31, 40, 1e-6, "c64")
    assert c.phi.shape == (31,) * 3 and np.count_nonzero(c.b) == 1
    s = I.small_2d()
    assert (s.n, s.k, s.tol, s.precision) == (127, 20.0, 1e-8, "c128")
    assert abs(s.k / (s.n + 1) - 0.156) < 0.001          # kh ~ 0.16
    w = I.large_2d(0.2)
    assert (w.n, w.k, w.theta_beta, w.tol) == (1023, 160.0, 0.2, 1e-6)
    assert abs(w.k / (w.n + 1) - 0.156) < 0.001
    assert I.LARGE_2D_BETAS == (0.1, 0.2, 0.3, 0.5)


def test_batch_sizes_and_wavenumbers():
    ws = I.batch_2d()
    assert len(ws) == 64
    assert {w.n for w in ws} == {255, 511, 1023}
    kh = np.array([w.k / (w.n + 1) for w in ws])
    assert kh.min() >= 0.1 and kh.max() <= 0.3
    assert all(w.theta_beta == 0.3 and w.restart == 40 and w.tol == 1e-6 for w in ws)
    assert all(w.b.shape == (w.n, w.n) for w in ws)


@pytest.mark.parametrize("count,rate", [(2000, 200.0), (120, 8.0)])
def test_request_stream_is_poisson_over_the_five_shapes(count, rate):
    st = I.request_stream(count=count, rate=rate)
    t = np.array([r.arrival for r in st])
    assert len(st) == count and np.all(np.diff(t) > 0) and t[0] > 0
    gaps = np.diff(np.concatenate(([0.0], t)))
    # exponential gaps: mean 1/rate, coefficient of variation 1 (loose bounds for 120)
    tol = 0.1 if count >= 2000 else 0.3
    assert abs(gaps.mean() * rate - 1.0) < tol
    assert abs(gaps.std() / gaps.mean() - 1.0) < tol
    shapes = {(r.work.dim, r.work.n) for r in st}
    assert shapes == {(2, 127), (2, 511), (2, 1023), (3, 127), (3, 255)}
    kh = np.array([r.work.k / (r.work.n + 1) for r in st])
    assert kh.min() >= 0.1 and kh.max() <= 0.3
    assert all(r.work.tol == 1e-6 and r.work.restart == 40 for r in st)
