"""Pins of the IMPES oracle (oracle/impes.py), CPU only: closed forms of the
mobilities, finite differences of the fractional-flow slope, the Welge
tangent, exact water balance of the transport step, the maximum principle
under the CFL limit, and the Buckley-Leverett front of a one-dimensional
displacement."""

import numpy as np

from oracle import impes as M
from oracle.fine import Grid, solve_direct, split_faces
from paper_1807_07220_gb300.inputs import channel_field, random_pairs


def test_mobility_closed_forms():
    for mw, mo in ((1.0, 5.0), (0.5, 2.0)):
        assert M.total_mobility(0.0, mw, mo) == 1.0 / mo and M.total_mobility(1.0, mw, mo) == 1.0 / mw
        assert M.frac_flow(0.0, mw, mo) == 0.0 and M.frac_flow(1.0, mw, mo) == 1.0
        # s = 1/2: f_w = mo / (mo + mw)
        assert abs(M.frac_flow(0.5, mw, mo) - mo / (mo + mw)) < 1e-15
        s = np.linspace(0.01, 0.99, 50)
        e = 1e-6
        fd = (M.frac_flow(s + e, mw, mo) - M.frac_flow(s - e, mw, mo)) / (2 * e)
        np.testing.assert_allclose(M.frac_flow_slope(s, mw, mo), fd, rtol=1e-8)


def test_welge_tangent():
    s_star, speed = M.welge_front()
    # mu_w = 1, mu_o = 5: f_w / s is largest where 1.2 s^2 = 0.2, s* = 6^{-1/2},
    # and there the line from the origin touches f_w
    exact = 6 ** -0.5
    assert abs(M.frac_flow_slope(exact) - M.frac_flow(exact) / exact) < 1e-13
    assert abs(s_star - exact) < 1e-5
    assert abs(speed - M.frac_flow(exact) / exact) < 1e-9
    s = np.linspace(1e-3, 1.0, 1000)
    assert np.all(M.frac_flow(s) <= speed * s + 1e-12)                      # the line stays above f_w


def _field(n, seed):
    g = Grid(n, 4)
    kap = channel_field(n, 1e3, seed)
    f = random_pairs(n, 2, seed)
    u, _ = solve_direct(g, kap, f)
    ux, uy = split_faces(g, u)
    return g, f, ux, uy


def test_transport_conserves_water_exactly():
    n = 16
    g, f, ux, uy = _field(n, 3)
    rng = np.random.default_rng(0)
    s = rng.random((n, n))
    s1, dt = M.transport_step(n, s, ux, uy, f)
    h = 1.0 / n
    fw = M.frac_flow(s)
    source = dt * (h * h * np.maximum(f, 0).sum() + (fw * h * h * np.minimum(f, 0)).sum())
    change = h * h * (s1 - s).sum()
    assert abs(change - source) <= 1e-13 * max(abs(source), 1e-300)
    assert dt > 0


def test_maximum_principle_under_cfl():
    n = 16
    g, f, ux, uy = _field(n, 4)
    s = np.zeros((n, n))
    for _ in range(40):
        s, dt = M.transport_step(n, s, ux, uy, f, cfl=0.5)
        assert s.min() >= -1e-14 and s.max() <= 1 + 1e-14


def test_buckley_leverett_front():
    """kappa = 1, inflow u = 1 through the left side, outflow through the
    right: the velocity is uniform, u_x = 1, and the saturation is the 1-D
    Buckley-Leverett solution, a shock at x = f_w'(s*) t."""
    n = 64
    g = Grid(n, 8)
    bflux = np.concatenate([-np.ones(n), np.ones(n), np.zeros(2 * n)])
    u, _ = solve_direct(g, np.ones((n, n)), np.zeros((n, n)), bflux)
    ux, uy = split_faces(g, u)
    np.testing.assert_allclose(ux, 1.0, atol=1e-10)
    np.testing.assert_allclose(uy, 0.0, atol=1e-10)
    s = np.zeros((n, n))
    t, T = 0.0, 0.4
    while t < T:
        s, dt = M.transport_step(n, s, ux, uy, np.zeros((n, n)))
        t += dt
    s_star, speed = M.welge_front()
    profile = s.mean(axis=0)
    x = (np.arange(n) + 0.5) / n
    front = x[np.argmax(profile < 0.5 * s_star)]
    assert abs(front - speed * t) < 4.0 / n
    # water injected through the left side: t (unit flux through a unit edge)
    assert abs(s.sum() / n ** 2 - t) < 1e-12
