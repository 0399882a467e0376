"""Nested-dissection solve of the FP64 coarse system (TG_COARSE_SOLVER_ND)
against the oracle and against the dense coarse inverse (GPU).

The oracle solves the coarse problem of eq. coarsepre (and the coarse RT0
problem of the preprocessing, Section 3) by a dense direct solve of the
saddle-point form; the library's nested-dissection factor must give the same
coarse correction to rounding: 1e-9 relative against the oracle (the bar of
every FP64 operator), 1e-11 against the library's own dense inverse, and the
full solve within 1e-8 of the sparse direct solve at rtol 1e-12.
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.fine import Grid, solve_direct  # noqa: E402
from oracle.twogrid import TwoGridSolver  # noqa: E402
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


def psi_from_interior(n, v):
    full = np.zeros((n, n))
    full[1:, 1:] = v.reshape(n - 1, n - 1)
    return full


def interior_from_psi(n, full):
    return np.asarray(full).reshape(n, n)[1:, 1:].ravel()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def coarse_of(tg, s, n, rho):
    z = torch.zeros(n, n, dtype=torch.float64, device=DEV)
    tg.tg_apply_coarse(s.h, dev(psi_from_interior(n, rho)), z)
    return z.cpu().numpy()


# (n, b, field): 4 blocks per side (two strips, one separator row), 12 and 16
# blocks per side (several strips), channels and a log-normal field
ND_CASES = {
    "32x32_b8_channels": (32, 8, lambda n: inputs.channel_field(n, 1e4, 3)),
    "96x96_b8_channels": (96, 8, lambda n: inputs.channel_field(n, 1e6, 11)),
    "128x128_b8_grf_channels": (128, 8, lambda n: inputs.grf_channel_field(n, 1e6, 5)),
    "64x64_b4_lognormal": (64, 4, lambda n: inputs.lognormal_field(n, 7, sigma=2.0)),
}


@pytest.mark.parametrize("name", sorted(ND_CASES))
def test_nd_coarse_correction_and_preprocessing_match_the_oracle(tg, name):
    n, b, kf = ND_CASES[name]
    kappa = kf(n)
    o = TwoGridSolver(n, b, kappa, tol=10.0)
    s = tg.Solver(kappa, b, 10.0, coarse_solver="nd")
    sd = tg.Solver(kappa, b, 10.0, coarse_solver="dense")
    try:
        rng = np.random.default_rng(5)
        r = o.project(rng.standard_normal(o.If.size))
        got = o.C @ interior_from_psi(n, coarse_of(tg, s, n, o.C.T @ r))
        assert rel(got, o.coarse_correction(r)) < 1e-9, rel(got, o.coarse_correction(r))
        # the preprocessing's coarse RT0 solve takes the same solver: within
        # 1e-10 of the oracle, or (high-contrast fields, where the coarse
        # RT0 system's conditioning sets the rounding of any direct solve) no
        # further from it than the dense inverse
        f = inputs.random_pairs(n, 3, 7)
        F = (1.0 / n) ** 2 * f.ravel()
        ref = o.preprocess(F, np.zeros(o.If.size))
        err = {}
        for which, h in (("nd", s), ("dense", sd)):
            ux = torch.zeros(n, n + 1, dtype=torch.float64, device=DEV)
            uy = torch.zeros(n + 1, n, dtype=torch.float64, device=DEV)
            tg.tg_preprocess(h.h, dev(f), None, ux, uy)
            u = np.concatenate([ux.cpu().numpy().ravel(), uy.cpu().numpy().ravel()])
            assert np.abs(o.B @ u - F).max() <= 1e-12 * np.abs(F).max()
            err[which] = rel(u[o.If], ref)
        assert err["nd"] < max(1e-10, 2.0 * err["dense"]), err
        # full solve: the direct solve's answer, the oracle's iteration count
        f = inputs.quarter_five_spot(n)
        it, rep = s.solve(f, rtol=1e-12)
        assert rep.coarse_solver == 2 and rep.converged == 1
        u_ref, p_ref = solve_direct(Grid(n, b), kappa, f)
        got_u = np.concatenate([s.ux.cpu().numpy().ravel(), s.uy.cpu().numpy().ravel()])
        assert rel(got_u, u_ref) < 1e-8 and rel(s.p.cpu().numpy().ravel(), p_ref) < 1e-8
        it8, _ = s.solve(f, rtol=1e-8)
        assert abs(it8 - o.solve(f, rtol=1e-8)["iters"]) <= 1
    finally:
        s.close()
        sd.close()


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_nd_matches_the_dense_inverse(tg, prec):
    """256^2 with 8 x 8 blocks (32 blocks per side, about 1 000 coarse
    unknowns): the two coarse solvers give the same coarse correction to
    rounding and the same solve; the factor reads far fewer bytes."""
    n, b = 256, 8
    kappa = inputs.grf_channel_field(n, 1e6, 2)
    kw = dict(precision=prec, flexible=int(prec != "f64"))
    sd = tg.Solver(kappa, b, 10.0, coarse_solver="dense", **kw)
    sn = tg.Solver(kappa, b, 10.0, coarse_solver="nd", **kw)
    try:
        rng = np.random.default_rng(9)
        rho = rng.standard_normal((n - 1) ** 2)
        zd, zn = coarse_of(tg, sd, n, rho), coarse_of(tg, sn, n, rho)
        assert rel(zn, zd) < 1e-11, rel(zn, zd)
        f = inputs.random_pairs(n, 4, 3)
        itd, repd = sd.solve(f, rtol=1e-10)
        itn, repn = sn.solve(f, rtol=1e-10)
        assert repd.coarse_solver == 1 and repn.coarse_solver == 2
        assert repn.coarse_solve_mb < 0.25 * repd.coarse_solve_mb, (repn.coarse_solve_mb, repd.coarse_solve_mb)
        assert abs(itn - itd) <= 1, (itn, itd)
        assert rel(sn.p.cpu().numpy(), sd.p.cpu().numpy()) < 1e-8
        assert repn.max_div_error < 1e-12
    finally:
        sd.close()
        sn.close()


def test_nd_handle_after_kappa_update(tg):
    """tg_update_kappa with the frozen coarse basis: the dense handle updates
    its inverse by low rank, the nested-dissection handle forms its factor
    again; both then apply the same preconditioner and reach the direct
    solve of the new permeability."""
    n, b = 64, 8
    k0 = inputs.channel_field(n, 1e5, 1)
    k1 = k0.copy()
    k1[20:30, 10:40] *= 0.01
    s = tg.Solver(k0, b, 10.0, coarse_solver="nd")
    t = tg.Solver(k0, b, 10.0, coarse_solver="dense")
    try:
        f = inputs.quarter_five_spot(n)
        for h in (s, t):
            h.solve(f, rtol=1e-12)
            tg.tg_update_kappa(h.h, dev(k1), 0)
        it, rep = s.solve(f, rtol=1e-12)
        it2, rep2 = t.solve(f, rtol=1e-12)
        assert rep.coarse_solver == 2 and rep.update_rank[0] == -1 and rep2.coarse_solver == 1
        assert abs(it - it2) <= 1, (it, it2)
        u_ref, p_ref = solve_direct(Grid(n, b), k1, f)
        got_u = np.concatenate([s.ux.cpu().numpy().ravel(), s.uy.cpu().numpy().ravel()])
        assert rel(got_u, u_ref) < 1e-8 and rel(s.p.cpu().numpy().ravel(), p_ref) < 1e-8
    finally:
        s.close()
        t.close()


def test_nd_in_a_batch(tg):
    """Instances of a batch (one graph launch, lock-step right-hand sides)
    take the factor too and solve like single handles."""
    specs = [(64, 8, 1e4, 1), (96, 8, 1e6, 2)]
    nrhs = 2
    kappas = [inputs.channel_field(n, c, seed) for n, b, c, seed in specs]
    kd = [dev(k) for k in kappas]
    opts = tg.default_options(precision="f16", flexible=1, coarse_solver="nd")
    batch = tg.tg_setup_batch(kd, [s[0] for s in specs], [s[1] for s in specs], 10.0, nrhs, options=opts,
                              stream=torch.cuda.current_stream().cuda_stream)
    try:
        fs, outs = [], []
        for n, b, c, seed in specs:
            for r in range(nrhs):
                fs.append(inputs.random_pairs(n, 2, 10 * seed + r))
                outs.append([torch.zeros(*sh, dtype=torch.float64, device=DEV) for sh in ((n, n + 1), (n + 1, n), (n, n))])
        iters, status = tg.tg_solve_batch(batch, [dev(f) for f in fs], None, 1e-12, [o[0] for o in outs],
                                          [o[1] for o in outs], [o[2] for o in outs])
        assert (status == 0).all()
        j = 0
        for (n, b, c, seed), k in zip(specs, kappas):
            for r in range(nrhs):
                u_ref, p_ref = solve_direct(Grid(n, b), k, fs[j])
                got_u = np.concatenate([outs[j][0].cpu().numpy().ravel(), outs[j][1].cpu().numpy().ravel()])
                assert rel(got_u, u_ref) < 1e-8 and rel(outs[j][2].cpu().numpy().ravel(), p_ref) < 1e-8
                j += 1
    finally:
        tg.tg_destroy_batch(batch)


def test_invalid_coarse_solver_is_rejected(tg):
    kappa = inputs.channel_field(32, 1e4, 3)
    o = tg.default_options(coarse_solver=3)
    with pytest.raises(tg.TgmsError) as e:
        tg.tg_setup(dev(kappa), 32, 8, 10.0, options=o, stream=torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -1


def test_auto_choice_and_switch_to_dense_under_kappa_updates(tg):
    """TG_COARSE_SOLVER_AUTO: the dense inverse for at most 768 coarse
    unknowns, nested dissection above; a handle whose kappa is changed with
    its basis kept turns to the dense inverse at that call (formed in full)
    and takes low-rank updates after it, solving like a fresh dense handle
    updated the same way."""
    small = tg.Solver(inputs.channel_field(64, 1e4, 2), 16, 10.0)
    try:
        _, rep = small.solve(inputs.quarter_five_spot(64), rtol=1e-8)
        assert rep.coarse_solver == 1 and rep.coarse_unknowns <= 768
    finally:
        small.close()
    n, b = 128, 4   # 32 blocks per side: 961 nodal functions
    k0 = inputs.channel_field(n, 1e5, 4)
    f = inputs.quarter_five_spot(n)
    s = tg.Solver(k0, b, 10.0, precision="f16", flexible=1)
    t = tg.Solver(k0, b, 10.0, precision="f16", flexible=1, coarse_solver="dense")
    try:
        _, rep = s.solve(f, rtol=1e-8)
        assert rep.coarse_solver == 2 and rep.coarse_unknowns > 768
        k = k0.copy()
        for step, (i0, j0) in enumerate(((62, 62), (25, 100))):
            k[j0:j0 + 4, i0:i0 + 4] *= 0.1
            for h in (s, t):
                tg.tg_update_kappa(h.h, dev(k), 0)
            it, rep = s.solve(f, rtol=1e-12)
            it2, rep2 = t.solve(f, rtol=1e-12)
            assert rep.coarse_solver == 1
            if step == 0:
                assert rep.update_rank[0] == -1 and rep.update_rank[1] == -1
            else:
                assert rep.update_rank[0] > 0 and rep.update_rank[1] > 0
            assert abs(it - it2) <= 1, (it, it2)
            u_ref, p_ref = solve_direct(Grid(n, b), k, f)
            got_u = np.concatenate([s.ux.cpu().numpy().ravel(), s.uy.cpu().numpy().ravel()])
            assert rel(got_u, u_ref) < 1e-8 and rel(s.p.cpu().numpy().ravel(), p_ref) < 1e-8
    finally:
        s.close()
        t.close()
