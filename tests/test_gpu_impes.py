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


def _rect_hits(rects, cells):
    """Rectangles (x0, y0, x1, y1), cell bounds inclusive, that hold a cell of `cells`."""
    return sum(any(x0 <= i <= x1 and y0 <= j <= y1 for i, j in cells) for x0, y0, x1, y1 in rects)


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_update_kappa_refactors_only_changed(tg, prec):
    """A permeability change confined to a few cells refactors only the
    patches and blocks holding one of them (patch K_i^+ of block (I, J) spans
    cells max(0, Ib - 2) .. min(n, (I + 1) b + 2) - 1 in each direction), and
    the updated handle's smoother, coarse space and solve agree with a fresh
    setup on the new permeability."""
    n, b, ov = 48, 8, 2
    nc = n // b
    k1 = inputs.lognormal_field(n, 3, sigma=1.0)
    k2 = k1.copy()
    cells = [(6, 0), (6, 1), (20, 33)]          # (i, j)
    for i, j in cells:
        k2[j, i] *= 7.0
    k2[40, 40] = k1[40, 40]                     # rewritten with the same value: no change
    patches = [(max(0, I * b - ov), max(0, J * b - ov), min(n, (I + 1) * b + ov) - 1, min(n, (J + 1) * b + ov) - 1)
               for J in range(nc) for I in range(nc)]
    blocks = [(I * b, J * b, I * b + b - 1, J * b + b - 1) for J in range(nc) for I in range(nc)]
    f = inputs.quarter_five_spot(n)
    opts = dict(precision=prec, flexible=int(prec != "f64"), smoother_shape=0)
    s = tg.Solver(dev(k1), b, 10.0, **opts)
    fresh = tg.Solver(dev(k2), b, 10.0, **opts)
    try:
        s.solve(f, rtol=1e-10)
        tg.tg_update_kappa(s.h, dev(k2), 1)
        it, rep = s.solve(f, rtol=1e-12)
        assert rep.refactored_patches == _rect_hits(patches, cells) == 4
        assert rep.refactored_blocks == _rect_hits(blocks, cells) == 2
        it_f, rep_f = fresh.solve(f, rtol=1e-12)
        assert rep_f.refactored_patches == nc * nc and it == it_f
        got = np.concatenate([s.ux.cpu().numpy().ravel(), s.uy.cpu().numpy().ravel()])
        ref = np.concatenate([fresh.ux.cpu().numpy().ravel(), fresh.uy.cpu().numpy().ravel()])
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
        rng = np.random.default_rng(5)
        rho = np.zeros((n, n))
        rho[1:, 1:] = rng.standard_normal((n - 1, n - 1))
        outs = []
        for sol in (s, fresh):
            for fn in (tg.tg_apply_smoother, tg.tg_apply_coarse):
                z = torch.zeros(n, n, dtype=torch.float64, device=DEV)
                fn(sol.h, dev(rho), z)
                outs.append(z.cpu().numpy())
        tol = 1e-13 if prec == "f64" else 1e-6     # same stored inverses; FP32 summation order for FP16
        for a, r in zip(outs[:2], outs[2:]):
            assert np.linalg.norm(a - r) <= tol * np.linalg.norm(r)
        # unchanged permeability: nothing refactored, same iterations
        tg.tg_update_kappa(s.h, dev(k2), 0)
        it2, rep2 = s.solve(f, rtol=1e-12)
        assert rep2.refactored_patches == 0 and rep2.refactored_blocks == 0 and it2 == it
    finally:
        s.close()
        fresh.close()


def test_low_rank_coarse_update_matches_full_inverse(tg):
    """A sequence of local permeability changes: the coarse inverses updated
    by low-rank corrections (coarse = 0) apply as the ones recomputed in full
    (coarse = 2), and the solves take the same iterations."""
    n, b = 64, 8
    rng = np.random.default_rng(11)
    k = inputs.channel_field(n, 1e4, 6)
    f = inputs.quarter_five_spot(n)
    lo = tg.Solver(dev(k), b, 10.0)
    full = tg.Solver(dev(k), b, 10.0)
    try:
        for step in range(6):
            k = k.copy()
            j0, i0 = rng.integers(0, n - 6, size=2)
            k[j0:j0 + 5, i0:i0 + 5] *= rng.uniform(0.2, 5.0, size=(5, 5))   # a 5 x 5 cell change
            tg.tg_update_kappa(lo.h, dev(k), 0)
            tg.tg_update_kappa(full.h, dev(k), 2)
            it, rep = lo.solve(f, rtol=1e-12)
            it_f, rep_f = full.solve(f, rtol=1e-12)
            assert 0 < rep.update_rank[0] and 4 * rep.update_rank[0] <= rep.coarse_unknowns, rep.update_rank
            assert 0 < rep.update_rank[1], rep.update_rank
            assert list(rep_f.update_rank) == [-1, -1]
            assert abs(it - it_f) <= 1
            rho = np.zeros((n, n))
            rho[1:, 1:] = rng.standard_normal((n - 1, n - 1))
            z = [torch.zeros(n, n, dtype=torch.float64, device=DEV) for _ in range(2)]
            tg.tg_apply_coarse(lo.h, dev(rho), z[0])
            tg.tg_apply_coarse(full.h, dev(rho), z[1])
            a, r = z[0].cpu().numpy(), z[1].cpu().numpy()
            assert np.linalg.norm(a - r) <= 1e-10 * np.linalg.norm(r), step
            got = np.concatenate([lo.ux.cpu().numpy().ravel(), lo.uy.cpu().numpy().ravel()])
            ref = np.concatenate([full.ux.cpu().numpy().ravel(), full.uy.cpu().numpy().ravel()])
            assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
        tg.tg_update_kappa(lo.h, dev(k), 0)                 # no change: nothing to update
        _, rep = lo.solve(f, rtol=1e-12)
        assert list(rep.update_rank) == [0, 0]
        with pytest.raises(tg.TgmsError):
            tg.tg_update_kappa(lo.h, dev(k), 3)
    finally:
        lo.close()
        full.close()


@pytest.mark.parametrize("prec,coarse", [("f64", "frozen"), ("f64", "frozen_full"), ("f64", "rebuild"),
                                        ("f64", "rebuild_learned"), ("bf16", "frozen")])
def test_impes_matches_oracle(tg, prec, coarse):
    """IMPES on the GPU against the oracle's IMPES on direct solves; the
    learned rebuild uses an untrained network (seeded initial weights), so
    its faces mostly fall back to the exact problem."""
    from paper_1807_07220_gb300.impes import Impes
    n, b, steps = 32, 8, 6
    g = Grid(n, b)
    kap = inputs.channel_field(n, 1e3, 4)
    f = inputs.quarter_five_spot(n)
    hist, dts = M.impes(g, kap, f, np.zeros((n, n)), steps, cfl=0.5)
    net = None
    opts = dict(coarse=coarse)
    if coarse == "rebuild_learned":
        din, dout, _ = tg.tg_mlp_shape(b, 4, 64)
        params = torch.as_tensor(inputs.mlp_init_params(din, dout, 64, 3), dtype=torch.float32, device=DEV)
        net = tg.Mlp(b, 4, 64, params, stream=stream())
        opts = dict(coarse="rebuild", coarse_space="learned", net=net)
    sim = Impes(dev(kap), dev(f), b, rtol=1e-12, precision=prec, flexible=int(prec != "f64"), **opts)
    try:
        for k in range(steps):
            dt, it = sim.step()
            assert abs(dt - dts[k]) <= 1e-9 * dts[k]
            np.testing.assert_allclose(sim.s.cpu().numpy(), hist[k + 1], rtol=0, atol=1e-9)
        assert sim.s.cpu().numpy().max() > 0.1       # water has entered
        if net is not None:
            assert all(h[7] > 0 for h in sim.history)   # the space was rebuilt every step
    finally:
        sim.close()
        if net is not None:
            net.close()
