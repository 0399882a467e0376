"""Learned coarse basis on the GPU against the FP64 oracle (oracle/learned.py).

* training data: face inputs bit-exact (bfloat16), spectra and selections of
  the exact problems, label projectors;
* network: forward pass and gradients against the oracle with the kernels'
  bfloat16 rounding points emulated (tight) and in plain FP64 (bfloat16
  accuracy), one Adam step;
* coarse space from given predicted profiles: selection, Ritz values,
  fallbacks and PCG iterations against the oracle's learned space, solution
  against the direct solve;
* end to end: a network trained on the GPU by the library's own kernels on
  fields of the benchmark's family, evaluated on a held-out field against the
  exact spectral space, the MsFEM space and the untrained network.
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import learned as L  # noqa: E402
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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def stream():
    return torch.cuda.current_stream().cuda_stream


def face_data(tg, kap, n, b, tol, k):
    nc = n // b
    F = 2 * nc * (nc - 1)
    din = (b + 2) * (2 * b + 2)
    x = torch.empty((F, din), dtype=torch.bfloat16, device=DEV)
    q = torch.empty((F, k, b), dtype=torch.float32, device=DEV)
    ns = torch.empty(F, dtype=torch.int32, device=DEV)
    la = torch.empty((F, b), dtype=torch.float64, device=DEV)
    tg.tg_face_data(dev(kap), n, b, tol, k, x, q, ns, la, stream=stream())
    return x, q, ns, la


def test_face_data_matches_oracle(tg):
    n, b, k, tol = 32, 8, 4, 10.0
    kap = inputs.channel_field(n, 1e4, 9, background=inputs.lognormal_field(n, 9, sigma=1.0))
    X, Q, nsel, lam = L.exact_profiles(Grid(n, b), kap, tol, k)
    x, q, ns, la = face_data(tg, kap, n, b, tol, k)
    np.testing.assert_array_equal(x.float().cpu().numpy(), L.bf16(X))
    np.testing.assert_allclose(la.cpu().numpy(), lam, rtol=1e-9)
    assert list(ns.cpu().numpy()) == list(nsel)
    qg = q.cpu().numpy().astype(np.float64)
    for f in range(len(X)):
        np.testing.assert_allclose(qg[f].T @ qg[f], Q[f].T @ Q[f], atol=2e-6)


def net_case(seed, b=8, k=4, hidden=64, batch=100):
    R, C = L.input_shape(b)
    din, dout = R * C, k * b
    rng = np.random.default_rng(seed)
    params = inputs.mlp_init_params(din, dout, hidden, seed).astype(np.float64)
    _, total = L.param_layout(b, k, hidden)
    p = L.unpack(params, b, k, hidden)
    for name in ("b1", "b2", "b3"):
        p[name] = 0.1 * rng.standard_normal(p[name].shape)
    params = L.pack(p, b, k, hidden).astype(np.float32)
    X = L.bf16(0.7 * rng.standard_normal((batch, din)))
    Q = np.zeros((batch, k, b))
    for s in range(batch):
        m = 1 + s % k
        Q[s, :m] = np.linalg.qr(rng.standard_normal((b, m)))[0].T
    return b, k, hidden, params, X, Q.astype(np.float32)


def test_forward_matches_oracle(tg):
    b, k, hidden, params, X, _ = net_case(1)
    net = tg.Mlp(b, k, hidden, dev(params, torch.float32), stream=stream())
    y = torch.empty((X.shape[0], k * b), dtype=torch.float32, device=DEV)
    net.forward(dev(X, torch.bfloat16), y)
    yg = y.cpu().numpy().astype(np.float64)
    p = L.unpack(params.astype(np.float64), b, k, hidden)
    ye, _ = L.forward(p, X, emulate_bf16=True)
    y64, _ = L.forward(p, X, emulate_bf16=False)
    assert rel(yg, ye) < 2e-3
    assert rel(yg, y64) < 3e-2
    net.close()


def test_gradients_match_oracle(tg):
    """Gradients of the subspace loss from the library's backward kernels
    against the FP64 oracle: with the kernels' bfloat16 rounding points
    emulated, and against the plain FP64 chain rule."""
    b, k, hidden, params, X, Q = net_case(2)
    net = tg.Mlp(b, k, hidden, dev(params, torch.float32), stream=stream())
    grad = torch.empty(params.size, dtype=torch.float32, device=DEV)
    loss = net.loss_grad(dev(X, torch.bfloat16), dev(Q, torch.float32), grad)
    gg = grad.cpu().numpy().astype(np.float64)
    le, ge = L.loss_and_grad(params.astype(np.float64), X, Q.astype(np.float64), b, k, hidden, emulate_bf16=True)
    l64, g64 = L.loss_and_grad(params.astype(np.float64), X, Q.astype(np.float64), b, k, hidden)
    assert abs(loss - le) <= 2e-3 * le
    assert abs(loss - l64) <= 3e-2 * l64
    layout, _ = L.param_layout(b, k, hidden)
    # The emulated comparison is the tight one.  Against plain FP64 the
    # bfloat16 weights move pre-activations near zero across the ReLU kink,
    # which switches whole units in or out of a sample's gradient: a few
    # percent, bounded here at 10%.
    for name, shp, off, size in layout:
        sl = slice(off, off + size)
        assert rel(gg[sl], ge[sl]) < 1e-2, name
        assert rel(gg[sl], g64[sl]) < 1e-1, name
    net.close()


def test_adam_step_matches_oracle(tg):
    b, k, hidden, params, X, Q = net_case(3)
    lr = 1e-3
    net = tg.Mlp(b, k, hidden, dev(params, torch.float32), stream=stream())
    order = torch.arange(X.shape[0], dtype=torch.int32, device=DEV)
    hist = torch.zeros(1, dtype=torch.float32, device=DEV)
    net.train(dev(X, torch.bfloat16), dev(Q, torch.float32), order, 1, X.shape[0], lr, hist)
    p1 = torch.empty(params.size, dtype=torch.float32, device=DEV)
    net.params(p1)
    dg = p1.cpu().numpy().astype(np.float64) - params.astype(np.float64)
    le, ge = L.loss_and_grad(params.astype(np.float64), X, Q.astype(np.float64), b, k, hidden, emulate_bf16=True)
    po, _, _ = L.adam_step(params.astype(np.float64), ge, np.zeros_like(ge), np.zeros_like(ge), 1, lr)
    do = po - params.astype(np.float64)
    big = np.abs(ge) > 1e-2 * np.abs(ge).max()          # signs of these gradients are unambiguous
    assert big.sum() > 100
    np.testing.assert_allclose(dg[big], do[big], atol=2e-3 * lr + 1e-7)
    assert np.abs(dg).max() <= lr * 1.001 + 1e-7
    assert abs(float(hist[0]) - le) <= 2e-3 * le
    net.close()


@pytest.mark.parametrize("mode", ["noisy_labels", "zeros"])
def test_learned_space_matches_oracle(tg, mode):
    n, b, k, tol = 32, 8, 4, 10.0
    kap = inputs.channel_field(n, 1e4, 9, background=inputs.lognormal_field(n, 9, sigma=1.0))
    g = Grid(n, b)
    _, Q, nsel_exact, _ = L.exact_profiles(g, kap, tol, k)
    F = len(Q)
    rng = np.random.default_rng(5)
    if mode == "zeros":
        prof = np.zeros((F, k, b), dtype=np.float32)
    else:
        prof = (Q + 0.05 * rng.standard_normal(Q.shape)).astype(np.float32)
    pd = dev(prof, torch.float32)
    solver = tg.Solver(dev(kap), b, tol, coarse_space="learned", face_profiles=pd, learned_k=k)
    nsel, lam, vb = tg.tg_coarse_info(solver.h, b)
    ora = TwoGridSolver(n, b, kap, tol=tol, coarse="learned", profiles=[prof[f].T.astype(np.float64) for f in range(F)])
    assert list(nsel) == list(ora.info["nsel"])
    f_src = inputs.random_pairs(n, 2, 4)
    it, rep = solver.solve(f_src, rtol=1e-12)
    assert rep.fallback_faces == int(np.sum(ora.info["fallback"]))
    if mode == "zeros":
        assert rep.fallback_faces == F and list(nsel) == list(nsel_exact)
    lam = np.asarray(lam).reshape(F, b)
    for f in range(F):
        ol = np.asarray(ora.info["lam"][f])
        np.testing.assert_allclose(lam[f, :ol.size], ol, rtol=1e-8)
    oit = ora.solve(f_src, rtol=1e-12)["iters"]
    assert abs(it - oit) <= 1
    ud, pdir = solve_direct(g, kap, f_src)
    ux, uy, p = solver.ux.cpu().numpy(), solver.uy.cpu().numpy(), solver.p.cpu().numpy()
    u = np.concatenate([ux.ravel(), uy.ravel()])
    assert rel(u, ud) < 1e-8
    assert rel(p.ravel(), pdir) < 1e-8
    solver.close()


def test_trained_network_against_exact_msfem_and_untrained(tg):
    """Train on 48 fields of the benchmark family (exp(GRF) + channels at 1e6,
    128 x 128, 16 x 16 blocks) with the library's kernels, then solve a
    held-out field with the learned space and compare with the exact spectral
    space, the MsFEM space and the untrained network."""
    n, b, k, hidden, tol = 128, 16, 4, 256, 10.0
    xs, qs = [], []
    for seed in range(48):
        kap = inputs.grf_channel_field(n, 1e6, 100 + seed)
        x, q, _, _ = face_data(tg, kap, n, b, tol, k)
        xs.append(x)
        qs.append(q)
    X = torch.cat(xs).contiguous()
    Qt = torch.cat(qs).contiguous()
    R, C = L.input_shape(b)
    params0 = inputs.mlp_init_params(R * C, k * b, hidden, 7)
    p0 = dev(params0, torch.float32)
    net = tg.Mlp(b, k, hidden, p0, stream=stream())
    untrained = tg.Mlp(b, k, hidden, p0, stream=stream())
    nsteps, batch = 1500, 256
    order = dev(inputs.sample_order(X.shape[0], nsteps, batch, 11), torch.int32)
    hist = torch.zeros(nsteps, dtype=torch.float32, device=DEV)
    net.train(X, Qt, order, nsteps, batch, 1e-3, hist)
    h = hist.cpu().numpy()
    print("loss: first %.4f last %.4f" % (h[:20].mean(), h[-100:].mean()))
    assert h[-100:].mean() < 0.5 * h[:20].mean()

    kap = inputs.grf_channel_field(n, 1e6, 999)
    f = inputs.quarter_five_spot(n)
    kd = dev(kap)
    out = {}
    for name, kw in (("exact", dict(coarse_space="gmsfem")), ("msfem", dict(coarse_space="msfem")),
                     ("learned", dict(coarse_space="learned", net=net)),
                     ("untrained", dict(coarse_space="learned", net=untrained))):
        s = tg.Solver(kd, b, tol, precision="f32", flexible=1, **kw)
        it, rep = s.solve(f, rtol=1e-8)
        out[name] = dict(iters=it, solves=rep.snapshot_solves, fallback=rep.fallback_faces,
                         basis=rep.velocity_basis, u=np.concatenate([s.ux.cpu().numpy().ravel(),
                                                                     s.uy.cpu().numpy().ravel()]))
        s.close()
    for name, v in out.items():
        print(name, {k2: v2 for k2, v2 in v.items() if k2 != "u"})
    F = 2 * (n // b) * (n // b - 1)
    e, l, m, u = out["exact"], out["learned"], out["msfem"], out["untrained"]
    assert rel(l["u"], e["u"]) < 1e-5
    assert l["iters"] <= max(e["iters"] + 3, int(1.3 * e["iters"]))
    assert l["iters"] < m["iters"]
    assert l["fallback"] < F // 4
    assert l["solves"] < 0.6 * e["solves"]
    assert l["fallback"] <= u["fallback"]
    net.close()
    untrained.close()
