"""Two-phase IMPES on the GPU against the oracle (oracle/impes.py): the total
mobility and transport kernels on given velocities, tg_update_kappa against a
fresh setup and the direct solve, and whole IMPES runs against the oracle's
IMPES on direct solves."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import impes as M  # noqa: E402
from oracle.fine import Grid, solve_direct, split_faces  # noqa: E402
from paper_1807_07220_gb300 import inputs  # noqa: E402

DEV = "cuda"


@pytest.fixture(scope="module")
def tg():
    from paper_1807_07220_gb300 import build, tgms
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(tgms.LIB_PATH):
        build.build_library()
    tgms.lib()
    return tgms


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("boundary", ["no_flow", "inflow"])
def test_transport_and_mobility_match_oracle(tg, boundary):
    n = 24
    g = Grid(n, 8)
    kap = inputs.channel_field(n, 1e3, 5)
    if boundary == "no_flow":
        f = inputs.random_pairs(n, 2, 5)
        u, _ = solve_direct(g, kap, f)
    else:
        f = np.zeros((n, n))
        bflux = np.concatenate([-np.ones(n), np.ones(n), np.zeros(2 * n)])
        u, _ = solve_direct(g, kap, f, bflux)
    ux, uy = split_faces(g, u)
    rng = np.random.default_rng(2)
    s = rng.random((n, n))
    lam = dev(np.zeros((n, n)))
    tg.tg_total_mobility(dev(kap), dev(s), n, 1.0, 5.0, lam, stream())
    np.testing.assert_allclose(lam.cpu().numpy(), kap * M.total_mobility(s), rtol=1e-15)
    out = dev(np.zeros((n, n)))
    dt = tg.tg_transport_step(dev(s), dev(ux), dev(uy), dev(f), n, 0.5, 1.0, 5.0, out, stream=stream())
    ref, dt_ref = M.transport_step(n, s, ux, uy, f, cfl=0.5)
    assert abs(dt - dt_ref) <= 1e-14 * dt_ref
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-13)
    # a fixed time step is used as given
    dt2 = tg.tg_transport_step(dev(s), dev(ux), dev(uy), dev(f), n, 0.5, 1.0, 5.0, out, dt_fixed=0.5 * dt_ref,
                               stream=stream())
    ref2, _ = M.transport_step(n, s, ux, uy, f, dt=0.5 * dt_ref)
    assert dt2 == 0.5 * dt_ref
    np.testing.assert_allclose(out.cpu().numpy(), ref2, rtol=0, atol=1e-13)


@pytest.mark.parametrize("coarse", [0, 1])
def test_update_kappa(tg, coarse):
    n, b = 32, 8
    g = Grid(n, b)
    k1 = inputs.channel_field(n, 1e4, 3)
    k2 = inputs.lognormal_field(n, 7, sigma=1.5)
    f = inputs.quarter_five_spot(n)
    u2, p2 = solve_direct(g, k2, f)
    s = tg.Solver(dev(k1), b, 10.0)
    fresh = tg.Solver(dev(k2), b, 10.0)
    try:
        s.solve(f, rtol=1e-10)                        # the graphs exist before the update
        tg.tg_update_kappa(s.h, dev(k2), coarse)
        it, rep = s.solve(f, rtol=1e-12)
        got = np.concatenate([s.ux.cpu().numpy().ravel(), s.uy.cpu().numpy().ravel()])
        assert np.linalg.norm(got - u2) <= 1e-8 * np.linalg.norm(u2)
        assert np.linalg.norm(s.p.cpu().numpy().ravel() - p2) <= 1e-8 * np.linalg.norm(p2)
        it_f, _ = fresh.solve(f, rtol=1e-12)
        if coarse == 1:
            assert it == it_f
    finally:
        s.close()
        fresh.close()


@pytest.mark.parametrize("prec,coarse", [("f64", "frozen"), ("f64", "rebuild"), ("bf16", "frozen")])
def test_impes_matches_oracle(tg, prec, coarse):
    from paper_1807_07220_gb300.impes import Impes
    n, b, steps = 32, 8, 6
    g = Grid(n, b)
    kap = inputs.channel_field(n, 1e3, 4)
    f = inputs.quarter_five_spot(n)
    hist, dts = M.impes(g, kap, f, np.zeros((n, n)), steps, cfl=0.5)
    sim = Impes(dev(kap), dev(f), b, rtol=1e-12, coarse=coarse, precision=prec, flexible=int(prec != "f64"))
    try:
        for k in range(steps):
            dt, it = sim.step()
            assert abs(dt - dts[k]) <= 1e-9 * dts[k]
            np.testing.assert_allclose(sim.s.cpu().numpy(), hist[k + 1], rtol=0, atol=1e-9)
        assert sim.s.cpu().numpy().max() > 0.1       # water has entered
    finally:
        sim.close()
