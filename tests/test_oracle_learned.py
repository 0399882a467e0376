"""Pins of the learned-coarse-basis oracle (CPU only).

Each test ties oracle/learned.py to something other than itself: the
bfloat16 conversion and Adam of a library (torch on the CPU), central finite
differences, the reflection symmetry of the discrete problem, the min-max
characterisation of eigenvalues, and the exact spectral coarse space."""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.coarse import BlockSolvers, coarse_faces, snapshots, spectral_problem, solve_spectral
from oracle.fine import Grid, assemble, solve_direct
from oracle.twogrid import TwoGridSolver
from oracle import learned as L
from paper_1807_07220_gb300.inputs import channel_field, lognormal_field, mlp_init_params, random_pairs

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        # exact ties between two bfloat16 neighbours, both parities
                        1.0 + np.arange(1, 64) * 2.0 ** -8, -(3.0 + np.arange(1, 64) * 2.0 ** -7), [0.0, -0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(L.bf16(x), ref)


def _spectral(g, kap, face, blocks, A, B, tol):
    sup, val = snapshots(g, A, B, blocks, face)
    a, s = spectral_problem(g, A, B, 1.0 / kap, face, sup, val)
    return a, s, solve_spectral(a, s, tol)


def test_transposed_face_has_the_same_problem():
    """A horizontal coarse edge of kappa and the vertical edge of kappa^T that
    the diagonal reflection maps it to: same canonical input, same spectrum,
    same selected span in flux-profile coordinates (no sign change)."""
    n, b = 16, 4
    g = Grid(n, b)
    kap = lognormal_field(n, 3, sigma=2.0)
    kapT = kap.T.copy()
    A, B = assemble(g, kap)
    AT, BT = assemble(g, kapT)
    blocks, blocksT = BlockSolvers(g, A, B), BlockSolvers(g, AT, BT)
    for face in [f for f in coarse_faces(g) if f[0] == 1][:6]:
        _, I, J = face
        faceT = (0, J, I)
        np.testing.assert_array_equal(L.face_input(kap, g, face), L.face_input(kapT, g, faceT))
        a, s, (lam, c) = _spectral(g, kap, face, blocks, A, B, 30.0)
        aT, sT, (lamT, cT) = _spectral(g, kapT, faceT, blocksT, AT, BT, 30.0)
        np.testing.assert_allclose(a, aT, rtol=1e-14)
        np.testing.assert_allclose(s, sT, rtol=1e-10, atol=1e-12 * np.abs(s).max())
        np.testing.assert_allclose(lam, lamT, rtol=1e-10)
        P = c @ np.linalg.pinv(c)
        PT = cT @ np.linalg.pinv(cT)
        np.testing.assert_allclose(P, PT, atol=1e-9)


def test_face_input_geometry():
    """Row l + 1 of the canonical patch holds the cells next to fine face e_l;
    columns b and b + 1 are the two cells that share it (K^1 then K^2); the
    halo outside the domain repeats the edge cell."""
    n, b = 16, 4
    g = Grid(n, b)
    kap = lognormal_field(n, 5, sigma=1.5)
    R, C = L.input_shape(b)
    for face in coarse_faces(g):
        kind, I, J = face
        x = L.face_input(kap, g, face).reshape(R, C)
        for l in range(b):
            if kind == 0:
                left, right = kap[J * b + l, I * b - 1], kap[J * b + l, I * b]
            else:
                left, right = kap[J * b - 1, I * b + l], kap[J * b, I * b + l]
            assert x[l + 1, b] == np.log10(left) / 3.0 and x[l + 1, b + 1] == np.log10(right) / 3.0
        if kind == 0 and J == 0:
            np.testing.assert_array_equal(x[0], x[1])        # y = -1 clamps to y = 0
        if kind == 1 and I == g.nc - 1:
            np.testing.assert_array_equal(x[-1], x[-2])      # x = n clamps to x = n - 1


def test_loss_is_basis_invariant_and_zero_on_the_label():
    rng = np.random.default_rng(1)
    b, k, B = 8, 4, 6
    Q = np.zeros((B, k, b))
    for s in range(B):
        m = 1 + s % k
        Q[s, :m] = np.linalg.qr(rng.standard_normal((b, m)))[0].T
    Y = rng.standard_normal((B, k * b))
    loss, _ = L.subspace_loss(Y, Q, b, k)
    assert loss > 0
    # G -> G R, R orthogonal (a rotation with a sign flip and a permutation)
    R = np.linalg.qr(rng.standard_normal((k, k)))[0] @ np.diag([1, -1, 1, -1])[:, [2, 0, 3, 1]]
    G = Y.reshape(B, k, b).transpose(0, 2, 1)
    Y2 = (G @ R).transpose(0, 2, 1).reshape(B, k * b)
    assert abs(L.subspace_loss(Y2, Q, b, k)[0] - loss) <= 1e-12 * loss
    # the label itself (any orthonormal basis of the same span) has zero loss
    G0 = Q.transpose(0, 2, 1) @ R
    l0, d0 = L.subspace_loss(G0.transpose(0, 2, 1).reshape(B, k * b), Q, b, k)
    assert l0 < 1e-26 and np.abs(d0).max() < 1e-13
    # orthonormal G: the loss is the squared distance of the projectors
    Gs = np.linalg.qr(rng.standard_normal((b, k)))[0]
    Qs = Q[3].T
    ref = np.linalg.norm(Gs @ Gs.T - Qs @ Qs.T) ** 2
    assert abs(L.subspace_loss(Gs.T.reshape(1, k * b), Q[3:4], b, k)[0] - ref) <= 1e-12 * ref


def test_gradient_by_central_differences():
    b, k, hidden, B = 2, 2, 6, 5
    R, C = L.input_shape(b)
    din = R * C
    rng = np.random.default_rng(2)
    flat = mlp_init_params(din, k * b, hidden, 4).astype(np.float64)
    flat += 0.1 * rng.standard_normal(flat.size)                       # non-zero biases too
    X = rng.standard_normal((B, din))
    Q = np.zeros((B, k, b))
    for s in range(B):
        Q[s, :1] = np.linalg.qr(rng.standard_normal((b, 1)))[0].T
    loss, grad = L.loss_and_grad(flat, X, Q, b, k, hidden)
    eps = 1e-6
    fd = np.zeros_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = eps
        fd[i] = (L.loss_and_grad(flat + e, X, Q, b, k, hidden)[0] -
                 L.loss_and_grad(flat - e, X, Q, b, k, hidden)[0]) / (2 * eps)
    np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())


def test_adam_matches_torch():
    rng = np.random.default_rng(3)
    p = rng.standard_normal(50)
    tp = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in range(1, 6):
        g = rng.standard_normal(50)
        p, m, v = L.adam_step(p, g, m, v, t, 1e-2)
        opt.zero_grad()
        tp.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


@pytest.fixture(scope="module")
def channel_problem():
    n, b = 16, 4
    g = Grid(n, b)
    kap = channel_field(n, 1e4, 9, background=lognormal_field(n, 9, sigma=1.0))
    A, B = assemble(g, kap)
    return g, kap, A, B, BlockSolvers(g, A, B)


def test_ritz_on_the_exact_span_reproduces_the_selection(channel_problem):
    g, kap, A, B, blocks = channel_problem
    for face in coarse_faces(g):
        a, s, (lam, c) = _spectral(g, kap, face, blocks, A, B, 10.0)
        G = np.zeros((g.b, 4))
        G[:, :c.shape[1]] = np.linalg.qr(np.sqrt(a)[:, None] * c)[0]      # whitened coordinates
        rl, rc, fb = L.ritz_select(G, a, s, 10.0)
        m = c.shape[1]
        np.testing.assert_allclose(rl[:m], lam[:m], rtol=1e-9)
        assert rc.shape[1] == m and fb == (lam[0] >= 10.0)
        np.testing.assert_allclose(rc @ np.linalg.pinv(rc), c @ np.linalg.pinv(c), atol=1e-8)


def test_ritz_values_bound_the_eigenvalues_from_above(channel_problem):
    """Min-max: the i-th Ritz value on any subspace is >= the i-th eigenvalue."""
    g, kap, A, B, blocks = channel_problem
    rng = np.random.default_rng(4)
    for face in coarse_faces(g)[:8]:
        a, s, (lam, _) = _spectral(g, kap, face, blocks, A, B, 1e300)
        G = np.linalg.qr(rng.standard_normal((g.b, 3)))[0]     # every direction kept
        rl, _, _ = L.ritz_select(G, a, s, 1e300)
        assert rl.size == 3
        assert np.all(rl >= lam[:3] * (1 - 1e-10))
        Gg = G / np.sqrt(a)[:, None]                               # flux profiles of the span
        ref = sla.eigh(Gg.T @ (a[:, None] * Gg), Gg.T @ s @ Gg, eigvals_only=True)
        np.testing.assert_allclose(rl, np.sort(ref), rtol=1e-9)


def test_learned_space_from_exact_labels_matches_gmsfem(channel_problem):
    """Exact labels as predictions (k = b) give back the GMsFEM space: same
    selection, same PCG iteration count, solution equal to the direct solve;
    all-zero predictions fall back on every face and give the same again."""
    g, kap, A, B, blocks = channel_problem
    n, b = g.n, g.b
    X, Q, nsel, lam = L.exact_profiles(g, kap, 10.0, b)
    f = random_pairs(n, 2, 1)
    ref = TwoGridSolver(n, b, kap, tol=10.0)
    it0 = ref.solve(f, rtol=1e-12)["iters"]
    for prof, expect_fb in ((Q.transpose(0, 2, 1), False), (np.zeros((len(Q), b, b)), True)):
        sol = TwoGridSolver(n, b, kap, tol=10.0, coarse="learned", profiles=prof)
        assert sol.info["nsel"] == ref.info["nsel"]
        assert all(fb == (expect_fb or l[0] >= 10.0) for fb, l in zip(sol.info["fallback"], ref.info["lam"]))
        out = sol.solve(f, rtol=1e-12)
        u, p = out["u"], out["p"]
        assert out["iters"] == it0
        ud, pd = solve_direct(g, kap, f)
        assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)
        assert np.linalg.norm(p - pd) <= 1e-8 * np.linalg.norm(pd)
