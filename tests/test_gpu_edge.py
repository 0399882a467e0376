"""Degenerate and smallest configurations of the method against the FP64
oracle (GPU).

The grids here are the limits that the grid validation admits:
- the smallest coarse blocks (b = 2, two fine faces per coarse face, so each
  spectral problem of Section 4.2 is 2 x 2);
- the smallest coarse grid (n / b = 2: four blocks and one interior coarse
  node), also at the largest block size b = 16;
- oversampling 1 and 2 (Section 6).
At 4 x 4 with b = 2 and oversampling 2 every patch K_i^+ covers the whole
domain, so the smoother alone solves the system exactly and PCG stops after
one iteration (condition number 1), a case the oracle reproduces.

Each case solves the quarter five-spot at rtol 1e-12 and compares velocity
and pressure with the oracle's sparse direct solve of the saddle-point system
(relative error 1e-8, per-cell mass balance 1e-12). At the paper's rtol 1e-8
the FP64 iteration count is within one of the oracle's PCG and the Lanczos
condition estimate within 5 %. The mixed-precision preconditioners (BF16,
FP16, flexible CG) reach the same accuracy."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.fine import Grid, solve_direct  # noqa: E402
from oracle.twogrid import TwoGridSolver  # noqa: E402
from paper_1807_07220_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def tg():
    from paper_1807_07220_gb300 import build, tgms
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(tgms.LIB_PATH):
        build.build_library()
    tgms.lib()
    return tgms


def _channels(n):
    return inputs.channel_field(n, 1e6, 7)


def _lognormal(n):
    return inputs.lognormal_field(n, 3, sigma=2.0)


# name: (n, b, oversampling, field)
EDGE = {
    "n4_b2_ov2_whole_domain_patches": (4, 2, 2, _channels),
    "n4_b2_ov1": (4, 2, 1, _lognormal),
    "n6_b2_ov1": (6, 2, 1, _lognormal),
    "n12_b2_ov2": (12, 2, 2, _channels),
    "n8_b4_ov1": (8, 4, 1, _channels),
    "n32_b16_ov2_two_by_two_blocks": (32, 16, 2, _channels),
    "n32_b16_ov1_two_by_two_blocks": (32, 16, 1, _lognormal),
}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", params=sorted(EDGE))
def case(request):
    n, b, ov, field = EDGE[request.param]
    kappa = field(n)
    f = inputs.quarter_five_spot(n)
    u_ref, p_ref = solve_direct(Grid(n, b), kappa, f)
    ora = TwoGridSolver(n, b, kappa, tol=10.0, overlap=ov).solve(f, rtol=1e-8)
    return dict(n=n, b=b, ov=ov, kappa=kappa, f=f, u_ref=u_ref, p_ref=p_ref, ora=ora)


def _solve(tg, c, rtol, **opts):
    s = tg.Solver(c["kappa"], c["b"], 10.0, overlap=c["ov"], **opts)
    try:
        it, rep = s.solve(c["f"], rtol=rtol)
        torch.cuda.synchronize()
        u = np.concatenate([s.ux.cpu().numpy().ravel(), s.uy.cpu().numpy().ravel()])
        p = s.p.cpu().numpy().ravel()
    finally:
        s.close()
    return it, rep, u, p


def test_edge_fp64_against_oracle(tg, case):
    it, rep, u, p = _solve(tg, case, 1e-12)
    assert rep.converged == 1
    assert _rel(u, case["u_ref"]) < 1e-8, _rel(u, case["u_ref"])
    assert _rel(p, case["p_ref"]) < 1e-8, _rel(p, case["p_ref"])
    assert rep.max_div_error < 1e-12
    it8, rep8, _, _ = _solve(tg, case, 1e-8)
    ora = case["ora"]
    assert abs(it8 - ora["iters"]) <= 1, (it8, ora["iters"])
    assert abs(rep8.cond_estimate / ora["cond"] - 1) < 0.05, (rep8.cond_estimate, ora["cond"])


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_edge_mixed_precision(tg, case, prec):
    it, rep, u, p = _solve(tg, case, 1e-12, precision=prec, flexible=1)
    assert rep.converged == 1
    assert _rel(u, case["u_ref"]) < 1e-8, _rel(u, case["u_ref"])
    assert _rel(p, case["p_ref"]) < 1e-8, _rel(p, case["p_ref"])
    assert rep.max_div_error < 1e-12


def _batch_solve(tg, specs, fs, nrhs, prec, rtol):
    dev = "cuda"
    kd = [torch.as_tensor(field(n), dtype=torch.float64, device=dev).contiguous() for n, b, field in specs]
    opts = tg.default_options(precision=prec, flexible=int(prec != "f64"))
    stream = torch.cuda.current_stream().cuda_stream
    batch = tg.tg_setup_batch(kd, [s[0] for s in specs], [s[1] for s in specs], 10.0, nrhs, options=opts,
                              stream=stream)
    try:
        assert tg.tg_batch_size(batch) == (len(specs), nrhs)
        outs = [(torch.full((n, n + 1), 7.0, dtype=torch.float64, device=dev),
                 torch.full((n + 1, n), 7.0, dtype=torch.float64, device=dev),
                 torch.full((n, n), 7.0, dtype=torch.float64, device=dev)) for (n, b, _) in specs for _ in range(nrhs)]
        fd = [torch.as_tensor(f, dtype=torch.float64, device=dev).contiguous() for f in fs]
        iters, status = tg.tg_solve_batch(batch, fd, None, rtol, [o[0] for o in outs], [o[1] for o in outs],
                                          [o[2] for o in outs])
        torch.cuda.synchronize()
        return iters, status, [tuple(t.cpu().numpy() for t in o) for o in outs]
    finally:
        tg.tg_destroy_batch(batch)


def test_batch_of_one_problem(tg):
    """One instance with one right-hand side: the batch graph holds a single
    chain, and its result is the direct solution."""
    n, b = 4, 2
    f = inputs.quarter_five_spot(n)
    iters, status, outs = _batch_solve(tg, [(n, b, _channels)], [f], 1, "f64", 1e-12)
    assert (status == 0).all() and iters.shape == (1,)
    u_ref, p_ref = solve_direct(Grid(n, b), _channels(n), f)
    u = np.concatenate([outs[0][0].ravel(), outs[0][1].ravel()])
    assert _rel(u, u_ref) < 1e-8 and _rel(outs[0][2].ravel(), p_ref) < 1e-8


@pytest.mark.parametrize("prec", ["f64", "bf16"])
def test_batch_of_smallest_grids_with_a_zero_source(tg, prec):
    """The smallest grids, each size twice (the later instance of a size
    takes the smoother shape tuned for the first), three right-hand sides per
    instance in lock step, the middle one of every instance zero.  The zero
    chains stop at once with the exact zero solution while the others of
    their group iterate on; every other chain reaches the direct solution."""
    specs = [(4, 2, _channels), (32, 16, _lognormal), (12, 2, _channels), (4, 2, _lognormal),
             (8, 4, _channels), (32, 16, _channels), (12, 2, _lognormal)]
    nrhs = 3
    fs = []
    for i, (n, b, _) in enumerate(specs):
        for r in range(nrhs):
            fs.append(np.zeros((n, n)) if r == 1 else inputs.random_pairs(n, 1, 10 * i + r))
    iters, status, outs = _batch_solve(tg, specs, fs, nrhs, prec, 1e-12)
    assert (status == 0).all(), status
    j = 0
    for i, (n, b, field) in enumerate(specs):
        for r in range(nrhs):
            ux, uy, p = outs[j]
            if r == 1:
                assert iters[j] == 0
                assert not ux.any() and not uy.any() and not p.any()
            else:
                assert iters[j] > 0
                u_ref, p_ref = solve_direct(Grid(n, b), field(n), fs[j])
                u = np.concatenate([ux.ravel(), uy.ravel()])
                assert _rel(u, u_ref) < 1e-8, (i, r, _rel(u, u_ref))
                assert _rel(p.ravel(), p_ref) < 1e-8, (i, r)
            j += 1
