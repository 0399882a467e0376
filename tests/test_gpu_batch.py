"""Batched solves (one CUDA graph for many instances and right-hand sides)
against the oracle's direct solves and against single solves (GPU)."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.fine import Grid, solve_direct  # noqa: E402
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["f64", "bf16"])
def test_batch_matches_direct_and_single_solves(tg, prec):
    specs = [(32, 8, 1e4, 1), (24, 4, 1e6, 2), (48, 16, 1e5, 3)]
    nrhs = 2
    dev = "cuda"
    kappas = [inputs.channel_field(n, c, seed) for n, b, c, seed in specs]
    kd = [torch.as_tensor(k, dtype=torch.float64, device=dev).contiguous() for k in kappas]
    opts = tg.default_options(precision=prec, flexible=int(prec != "f64"))
    stream = torch.cuda.current_stream().cuda_stream
    batch = tg.tg_setup_batch(kd, [s[0] for s in specs], [s[1] for s in specs], 10.0, nrhs, options=opts,
                              stream=stream)
    try:
        assert tg.tg_batch_size(batch) == (len(specs), nrhs)
        fs, outs = [], []
        for (n, b, c, seed), k in zip(specs, kappas):
            for r in range(nrhs):
                f = inputs.random_pairs(n, 2, 100 * seed + r)
                fs.append(f)
                outs.append((torch.zeros(n, n + 1, dtype=torch.float64, device=dev),
                             torch.zeros(n + 1, n, dtype=torch.float64, device=dev),
                             torch.zeros(n, n, dtype=torch.float64, device=dev)))
        fd = [torch.as_tensor(f, dtype=torch.float64, device=dev).contiguous() for f in fs]
        for rep in range(2):   # the batch graph is replayed
            iters, status = tg.tg_solve_batch(batch, fd, None, 1e-12, [o[0] for o in outs], [o[1] for o in outs],
                                              [o[2] for o in outs])
            assert (status == 0).all() and (iters > 0).all()
        j = 0
        for (n, b, c, seed), k in zip(specs, kappas):
            s = tg.Solver(k, b, 10.0, precision=prec, flexible=int(prec != "f64"))
            try:
                for r in range(nrhs):
                    u_ref, p_ref = solve_direct(Grid(n, b), k, fs[j])
                    got_u = np.concatenate([outs[j][0].cpu().numpy().ravel(), outs[j][1].cpu().numpy().ravel()])
                    got_p = outs[j][2].cpu().numpy().ravel()
                    assert rel(got_u, u_ref) < 1e-8 and rel(got_p, p_ref) < 1e-8
                    it1, _ = s.solve(fs[j], rtol=1e-12)
                    assert abs(it1 - iters[j]) <= 1
                    j += 1
            finally:
                s.close()
    finally:
        tg.tg_destroy_batch(batch)


def _run_batch(tg, kd, specs, fs, nrhs, prec, lockstep, rtol, **extra):
    dev = "cuda"
    opts = tg.default_options(precision=prec, flexible=int(prec != "f64"), batch_lockstep=lockstep, **extra)
    stream = torch.cuda.current_stream().cuda_stream
    batch = tg.tg_setup_batch(kd, [s[0] for s in specs], [s[1] for s in specs], 10.0, nrhs, options=opts,
                              stream=stream)
    try:
        outs = [(torch.zeros(n, n + 1, dtype=torch.float64, device=dev),
                 torch.zeros(n + 1, n, dtype=torch.float64, device=dev),
                 torch.zeros(n, n, dtype=torch.float64, device=dev)) for (n, b, c, seed) in specs for _ in range(nrhs)]
        fd = [torch.as_tensor(f, dtype=torch.float64, device=dev).contiguous() for f in fs]
        iters, status = tg.tg_solve_batch(batch, fd, None, rtol, [o[0] for o in outs], [o[1] for o in outs],
                                          [o[2] for o in outs])
        assert (status == 0).all()
        return iters, [np.concatenate([o[0].cpu().numpy().ravel(), o[1].cpu().numpy().ravel()]) for o in outs]
    finally:
        tg.tg_destroy_batch(batch)


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_lockstep_groups_match_independent_chains(tg, prec):
    """Right-hand sides of an instance in lock step (groups of up to 4 sharing
    the smoother sweeps; 5 per instance makes a group of 4 and a lone chain)
    give the iteration counts and solutions of independent chains, and the
    direct solution; their different source pairs make the chains of a group
    stop at different iterations."""
    specs = [(32, 8, 1e4, 1), (48, 16, 1e5, 3)]
    nrhs = 5
    kappas = [inputs.channel_field(n, c, seed) for n, b, c, seed in specs]
    kd = [torch.as_tensor(k, dtype=torch.float64, device="cuda").contiguous() for k in kappas]
    fs = [inputs.random_pairs(n, 1 + r % 3, 50 * seed + r) for (n, b, c, seed) in specs for r in range(nrhs)]
    it_l, u_l = _run_batch(tg, kd, specs, fs, nrhs, prec, 1, 1e-12)
    it_i, u_i = _run_batch(tg, kd, specs, fs, nrhs, prec, 0, 1e-12)
    assert len(set(it_l.tolist())) > 1                 # the chains stop at different iterations
    assert np.abs(it_l - it_i).max() <= 1, (it_l, it_i)
    j = 0
    for (n, b, c, seed), k in zip(specs, kappas):
        for r in range(nrhs):
            u_ref, _ = solve_direct(Grid(n, b), k, fs[j])
            assert rel(u_l[j], u_ref) < 1e-8 and rel(u_i[j], u_ref) < 1e-8, (j, rel(u_l[j], u_ref))
            j += 1


def test_lockstep_batch_with_band_smoother(tg):
    """Lock-step groups whose handles use the band smoother (tile shape 7,
    one band sweep per chain inside the group) reach the direct solution."""
    specs = [(32, 8, 1e4, 1), (48, 16, 1e5, 3)]
    nrhs = 3
    kappas = [inputs.channel_field(n, c, seed) for n, b, c, seed in specs]
    kd = [torch.as_tensor(k, dtype=torch.float64, device="cuda").contiguous() for k in kappas]
    fs = [inputs.random_pairs(n, 1, 70 * seed + r) for (n, b, c, seed) in specs for r in range(nrhs)]
    it, u = _run_batch(tg, kd, specs, fs, nrhs, "f32", 1, 1e-12, smoother_shape=7)
    j = 0
    for (n, b, c, seed), k in zip(specs, kappas):
        for r in range(nrhs):
            u_ref, _ = solve_direct(Grid(n, b), k, fs[j])
            assert rel(u[j], u_ref) < 1e-8, (j, rel(u[j], u_ref))
            j += 1


def test_learned_batch_takes_the_network_of_each_block_size(tg):
    """A learned-coarse-space batch over instances of two block sizes takes,
    per instance, the network trained for its block size (batch_nets); the
    solutions reach the direct solve.  With no network for one of the block
    sizes the setup is rejected."""
    specs = [(32, 8, 1e4, 1), (48, 16, 1e5, 3), (32, 16, 1e6, 4)]
    nrhs = 2
    kappas = [inputs.channel_field(n, c, seed) for n, b, c, seed in specs]
    kd = [torch.as_tensor(k, dtype=torch.float64, device="cuda").contiguous() for k in kappas]
    fs = [inputs.random_pairs(n, 1, 90 * seed + r) for (n, b, c, seed) in specs for r in range(nrhs)]
    stream = torch.cuda.current_stream().cuda_stream
    nets = []
    try:
        for b in (16, 8):
            din, dout, npar = tg.tg_mlp_shape(b, 4, 64)
            params = torch.as_tensor(inputs.mlp_init_params(din, dout, 64, 17 + b), device="cuda")
            nets.append(tg.Mlp(b, 4, 64, params, stream=stream))
        it, u = _run_batch(tg, kd, specs, fs, nrhs, "f16", 1, 1e-12, coarse_space="learned", batch_nets=nets)
        j = 0
        for (n, b, c, seed), k in zip(specs, kappas):
            for r in range(nrhs):
                u_ref, _ = solve_direct(Grid(n, b), k, fs[j])
                assert rel(u[j], u_ref) < 1e-8, (j, rel(u[j], u_ref))
                j += 1
        with pytest.raises(tg.TgmsError) as e:
            _run_batch(tg, kd, specs, fs, nrhs, "f16", 1, 1e-12, coarse_space="learned", batch_nets=nets[:1])
        assert e.value.code == -1
    finally:
        for net in nets:
            net.close()


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_lockstep_tensor_core_smoother(tg, prec):
    """Lock-step groups on the tensor-core tiles (tile shape 8: one A load per
    tile for up to four chains, two chains per B operand): the iteration
    counts of independent chains and the direct solution, with five
    right-hand sides per instance (a group of four and a lone chain)."""
    specs = [(32, 8, 1e4, 1), (48, 16, 1e5, 3), (64, 16, 1e6, 5)]
    nrhs = 5
    kappas = [inputs.channel_field(n, c, seed) for n, b, c, seed in specs]
    kd = [torch.as_tensor(k, dtype=torch.float64, device="cuda").contiguous() for k in kappas]
    fs = [inputs.random_pairs(n, 1 + r % 3, 60 * seed + r) for (n, b, c, seed) in specs for r in range(nrhs)]
    it_l, u_l = _run_batch(tg, kd, specs, fs, nrhs, prec, 1, 1e-12, smoother_shape=8)
    it_i, u_i = _run_batch(tg, kd, specs, fs, nrhs, prec, 0, 1e-12, smoother_shape=8)
    assert np.abs(it_l - it_i).max() <= 1, (it_l, it_i)
    j = 0
    for (n, b, c, seed), k in zip(specs, kappas):
        for r in range(nrhs):
            u_ref, _ = solve_direct(Grid(n, b), k, fs[j])
            assert rel(u_l[j], u_ref) < 1e-8 and rel(u_i[j], u_ref) < 1e-8, (j, rel(u_l[j], u_ref))
            j += 1
