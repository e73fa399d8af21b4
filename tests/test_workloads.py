"""The seeded input generators against the workload recipes they claim:
Gaussian sources of unit mass, a Y-shaped waveguide with 3x contrast, a
stationary Gaussian-covariance random medium, the stated wavelength
resolutions, the batched sampler's ranges and the Poisson arrival stream.
No solver arithmetic is involved (the generators hold none)."""

import math

import numpy as np
import pytest

from workloads import configs, fields


def test_gaussian_source_has_unit_mass_and_its_width():
    w = 0.02
    g = np.linspace(-0.2, 0.2, 2001)
    X, Y = np.meshgrid(g, g)
    s = fields.gaussian_source(X + 0.3, Y + 0.6, (0.3, 0.6), w)
    h = g[1] - g[0]
    assert abs(s.sum() * h * h - 1.0) < 1e-9
    # second moment of a 2D Gaussian: E[x^2] = w^2
    assert abs((s * X * X).sum() * h * h - w * w) < 1e-9


def test_y_channel_geometry_and_contrast():
    g = np.linspace(0.0, 1.0, 1201)
    X, Y = np.meshgrid(g, g)
    c = fields.y_channel_speed(X, Y)
    assert set(np.unique(c)) == {1.0 / 3.0, 1.0}
    # area: stem (length 0.5) and two arms (length sqrt(0.3^2 + 0.5^2)) of
    # width 0.08, with round ends and overlaps at the junction of lower order
    frac = np.mean(c < 1.0)
    arm = math.hypot(0.3, 0.5)
    assert abs(frac - 0.08 * (0.5 + 2 * arm)) < 0.01
    # the stem's centre line is slow, points 0.05 beside it are not
    assert fields.y_channel_speed(np.array(0.5), np.array(0.25)) == pytest.approx(1 / 3)
    assert fields.y_channel_speed(np.array(0.55), np.array(0.25)) == 1.0
    # the arms end at (0.2, 1) and (0.8, 1)
    assert fields.y_channel_speed(np.array(0.2), np.array(0.99)) == pytest.approx(1 / 3)
    assert fields.y_channel_speed(np.array(0.8), np.array(0.99)) == pytest.approx(1 / 3)


def test_random_field_covariance_is_that_of_its_modes():
    """g = sqrt(2/K) sum_k cos(k.x + phi_k): its spatial covariance at lag r
    is (1/K) sum_k cos(k.r) for the drawn wave vectors (cross terms average
    out over a large window), and for k ~ N(0, I/corr_len^2) that sum
    estimates exp(-|r|^2 / (2 corr_len^2)) (0.607 at r = corr_len)."""
    ell, seed, K = 0.05, 3, 256
    rng = np.random.default_rng(seed)
    kx = rng.standard_normal(K) / ell  # first draw of the generator (the lag below is along x)
    n = 1600
    gx = np.linspace(-2.0, 2.0, n)
    gy = np.linspace(-2.0, 2.0, n)
    f = fields.random_field(gx, gy, ell, seed, n_modes=K)
    h = gx[1] - gx[0]
    assert abs(f.mean()) < 0.03
    assert abs(f.var() - 1.0) < 0.05
    for lag_nodes in (10, 20, 40):
        r = lag_nodes * h
        corr = np.mean(f[:, :-lag_nodes] * f[:, lag_nodes:]) / f.var()
        modes = np.mean(np.cos(kx * r))
        assert abs(corr - modes) < 0.03, (r, corr, modes)
        assert abs(modes - math.exp(-r * r / (2 * ell * ell))) < 0.08, (r, modes)


def test_random_speed_is_the_clipped_field():
    gx = np.linspace(-1, 1, 300)
    c = fields.random_speed(gx, gx, 0.05, 3)
    g = fields.random_field(gx, gx, 0.05, 3)
    np.testing.assert_array_equal(c, 1.0 + 0.5 * np.clip(g, -1.5, 1.5))
    assert c.min() >= 0.25 and c.max() <= 1.75
    assert 0.01 < np.mean(np.abs(g) > 1.5) < 0.3  # the clip is active but rare


def test_wavelength_resolution_of_the_benchmark_workloads():
    # 256^2 quads, P = 3 on the unit square: node spacing 1/768; slow medium c = 1/3
    w2 = configs.config2()
    h2 = (w2.box[1] - w2.box[0]) / (w2.nx * w2.P)
    slow = 2 * math.pi * (1 / 3) / w2.omega
    assert slow / h2 == pytest.approx(8.0)
    assert slow / w2.src_width > 3  # the source resolves the slow wavelength
    # 1024^2 quads, P = 4 on [-1, 1]^2: spacing 1/2048; c = 1
    w3 = configs.config3()
    h3 = (w3.box[1] - w3.box[0]) / (w3.nx * w3.P)
    assert (2 * math.pi / w3.omega) / h3 == pytest.approx(10.0)
    assert (w3.sub_nx * w3.P + 1) ** 2 == 16641 and w3.L == 1024
    assert (w2.sub_nx * w2.P + 1) ** 2 == 625 and w2.L == 1024
    w1 = configs.config1()
    assert w1.num_nodes == 4225 and w1.L == 16


def test_batched_sampler_ranges():
    ws = configs.config4()
    assert len(ws) == 64
    assert {w.nx for w in ws} <= {64, 128, 256, 512} and len({w.nx for w in ws}) >= 3
    assert {w.P for w in ws} == {2, 3, 4, 5}
    assert all(w.sub_nx in (4, 8, 16, 32) and w.sub_nx <= w.nx // 4 for w in ws)
    assert all(5.0 <= w.omega <= 80.0 for w in ws)
    assert {w.speed_kind for w in ws} == {"random", "channel"}
    assert all(0.2 <= w.src_center[0] <= 0.8 and 0.2 <= w.src_center[1] <= 0.8 for w in ws)
    # each source resolves a quarter of the slowest wavelength
    for w in ws:
        cmin = 0.25 if w.speed_kind == "random" else 1 / 3
        assert w.src_width <= 0.25 * 2 * math.pi * cmin / w.omega + 1e-15
    assert [w.name for w in configs.config4()] == [w.name for w in ws]  # seeded


def test_poisson_arrivals_rate_and_groups():
    arr = configs.config5_arrivals()
    assert len(arr) == 2000
    t = np.array([a[0] for a in arr])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # mean gap 1/200 s (standard error 1/(200 sqrt(2000)) = 1.1e-4 s)
    assert abs(gaps.mean() - 1 / 200) < 5e-4
    # exponential gaps: the coefficient of variation is 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    groups = np.mean([a[2] == 8 for a in arr])
    assert abs(groups - 0.2) < 0.03 and {a[2] for a in arr} == {1, 8}
    assert len({a[1].name for a in arr}) > 40  # drawn from the 64-problem pool
