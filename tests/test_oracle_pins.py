"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one part of the oracle to the mathematics or to the paper:
quadrature of the RT0 basis, closed-form discrete solutions, exact
identities (div curl = 0, mass conservation), a library eigensolver, brute
force on tiny grids, the O(h^2) superconvergence of RT0/P0, and the paper's
kappa == 1 worked example (Model 1, Tables 1-3: Cond 3.6, one basis function
per coarse face)."""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.fine import Grid, assemble, solve_direct, solve_direct_pinned, split_faces, curl_matrix, boundary_lift
from oracle.coarse import (BlockSolvers, coarse_faces, face_blocks, fine_faces_on, jacobi_eigh,
                           snapshots, spectral_problem, solve_spectral)
from oracle.twogrid import TwoGridSolver
from paper_1807_07220_gb300.inputs import channel_field, lognormal_field, random_pairs, quarter_five_spot


# --------------------------------------------------------------------- fine system
def test_mass_and_divergence_by_quadrature():
    """A_{fe} = int kappa^{-1} phi_f . phi_e and B_{cf} = int_c div phi_f,
    recomputed cell by cell with 3-point Gauss quadrature of the RT0 basis."""
    n = 3
    g = Grid(n, 1)
    kappa = lognormal_field(n, 7)
    A, B = assemble(g, kappa)
    h = g.h
    gx, gw = np.polynomial.legendre.leggauss(3)
    Aq = np.zeros((g.nf, g.nf))
    Bq = np.zeros((g.ncell, g.nf))
    for j in range(n):
        for i in range(n):
            x0, y0 = i * h, j * h
            faces = [g.xface(i, j), g.xface(i + 1, j), g.yface(i, j), g.yface(i, j + 1)]

            def basis(x, y):
                return [np.array([(x0 + h - x) / h, 0.0]), np.array([(x - x0) / h, 0.0]),
                        np.array([0.0, (y0 + h - y) / h]), np.array([0.0, (y - y0) / h])]
            for a, wa in zip(gx, gw):
                for bq, wb in zip(gx, gw):
                    x, y = x0 + h * (a + 1) / 2, y0 + h * (bq + 1) / 2
                    w = wa * wb * h * h / 4
                    ph = basis(x, y)
                    for p_ in range(4):
                        for q_ in range(4):
                            Aq[faces[p_], faces[q_]] += w / kappa[j, i] * ph[p_] @ ph[q_]
            # divergence of each local basis function is +-1/h, area h^2
            for f_, sgn in zip(faces, [-1, 1, -1, 1]):
                Bq[g.cell(i, j), f_] += sgn * h
    np.testing.assert_allclose(A.toarray(), Aq, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(B.toarray(), Bq, rtol=0, atol=1e-15)


def test_divergence_of_curl_is_zero():
    g = Grid(12, 4)
    _, B = assemble(g, np.ones((12, 12)))
    C = curl_matrix(g)
    BC = (B[:, g.interior_faces()] @ C).toarray()
    assert np.abs(BC).max() == 0.0


def _layered_case(n, rng):
    krow = np.exp(rng.standard_normal(n) * 2)
    kappa = np.repeat(krow[:, None], n, axis=1)
    bflux = np.concatenate([krow, -krow, np.zeros(n), np.zeros(n)])
    return kappa, bflux, krow


def test_layered_medium_closed_form():
    """kappa = kappa(y), p = x: u_x = -kappa(row), u_y = 0 exactly."""
    n, b = 16, 4
    g = Grid(n, b)
    kappa, bflux, krow = _layered_case(n, np.random.default_rng(1))
    f = np.zeros((n, n))
    xc = (np.arange(n) + 0.5) / n
    p_exact = np.tile(xc - xc.mean(), (n, 1))
    u, p = solve_direct(g, kappa, f, bflux)
    ux, uy = split_faces(g, u)
    np.testing.assert_allclose(ux, -np.repeat(krow[:, None], n + 1, axis=1), rtol=1e-11)
    assert np.abs(uy).max() < 1e-11 * krow.max()
    np.testing.assert_allclose(p.reshape(n, n), p_exact, atol=1e-11)
    out = TwoGridSolver(n, b, kappa, tol=10.0).solve(f, bflux, rtol=1e-13)
    ux2, uy2 = split_faces(g, out["u"])
    np.testing.assert_allclose(ux2, ux, rtol=1e-9, atol=1e-9 * krow.max())
    np.testing.assert_allclose(out["p"].reshape(n, n), p_exact, atol=1e-9)


def test_series_medium_closed_form():
    """kappa = kappa(x), uniform flux q: p_L - p_R = q h (1/kappa_L + 1/kappa_R)/2."""
    n, b = 16, 4
    g = Grid(n, b)
    rng = np.random.default_rng(2)
    kcol = np.exp(rng.standard_normal(n) * 2)
    kappa = np.repeat(kcol[None, :], n, axis=0)
    q = 0.7
    bflux = np.concatenate([np.full(n, -q), np.full(n, q), np.zeros(n), np.zeros(n)])
    u, p = solve_direct(g, kappa, np.zeros((n, n)), bflux)
    ux, uy = split_faces(g, u)
    np.testing.assert_allclose(ux, q, rtol=1e-10)
    assert np.abs(uy).max() < 1e-10
    drop = q * g.h * 0.5 * (1 / kcol[:-1] + 1 / kcol[1:])
    prow = np.concatenate([[0.0], -np.cumsum(drop)])
    prow -= prow.mean()
    np.testing.assert_allclose(p.reshape(n, n), np.tile(prow, (n, 1)), atol=1e-10 * np.abs(prow).max())


def test_mass_conservation_direct_pcg_and_preprocessing():
    n, b = 16, 4
    g = Grid(n, b)
    kappa = lognormal_field(n, 3, sigma=2.0)
    f = random_pairs(n, 3, 4)
    A, B = assemble(g, kappa)
    F = g.h ** 2 * f.ravel()
    u, p = solve_direct(g, kappa, f)
    assert np.abs(B @ u - F).max() <= 1e-12 * np.abs(F).max()
    s = TwoGridSolver(n, b, kappa, tol=10.0)
    out = s.solve(f, rtol=1e-10)
    assert np.abs(B @ out["u"] - F).max() <= 1e-12 * np.abs(F).max()
    assert np.abs(s.BI @ out["vbar"] - F).max() <= 1e-12 * np.abs(F).max()
    assert np.linalg.norm(out["u"] - u) <= 1e-8 * np.linalg.norm(u)
    assert np.linalg.norm(out["p"] - p) <= 1e-8 * np.linalg.norm(p)


def test_incompatible_source_is_rejected():
    n = 8
    f = np.zeros((n, n))
    f[0, 0] = 1.0
    with pytest.raises(ValueError):
        solve_direct(Grid(n, 4), np.ones((n, n)), f)
    with pytest.raises(ValueError):
        TwoGridSolver(n, 4, np.ones((n, n))).solve(f)


def test_brute_force_dense_saddle():
    """Dense least-squares solve of the singular (unbordered) saddle system,
    then mean-zero pressure, against the bordered sparse solve."""
    n = 4
    g = Grid(n, 2)
    kappa = lognormal_field(n, 5, sigma=1.5)
    f = random_pairs(n, 2, 6)
    A, B = assemble(g, kappa)
    I = g.interior_faces()
    AII, BI = A[I][:, I].toarray(), B[:, I].toarray()
    K = np.block([[AII, BI.T], [BI, np.zeros((n * n, n * n))]])
    rhs = np.concatenate([np.zeros(I.size), g.h ** 2 * f.ravel()])
    x = np.linalg.lstsq(K, rhs, rcond=None)[0]
    v, p_paper = x[: I.size], x[I.size:]
    p_phys = -(p_paper - p_paper.mean())
    u, p = solve_direct(g, kappa, f)
    np.testing.assert_allclose(u[I], v, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(p, p_phys, rtol=1e-10, atol=1e-14)


def test_pinned_direct_solve():
    """solve_direct_pinned (pressure constant fixed by a pinned cell, then
    mean zero) reproduces the layered closed form with prescribed boundary
    flux, the dense least-squares solution of the unbordered system, and the
    bordered solve on a high-contrast channel field with a source pair."""
    n, b = 16, 4
    g = Grid(n, b)
    kappa, bflux, krow = _layered_case(n, np.random.default_rng(1))
    xc = (np.arange(n) + 0.5) / n
    u, p = solve_direct_pinned(g, kappa, np.zeros((n, n)), bflux)
    ux, uy = split_faces(g, u)
    np.testing.assert_allclose(ux, -np.repeat(krow[:, None], n + 1, axis=1), rtol=1e-11)
    assert np.abs(uy).max() < 1e-11 * krow.max()
    np.testing.assert_allclose(p.reshape(n, n), np.tile(xc - xc.mean(), (n, 1)), atol=1e-11)
    # brute force: dense least squares of the singular saddle system
    n4 = 4
    g4 = Grid(n4, 2)
    k4 = lognormal_field(n4, 5, sigma=1.5)
    f4 = random_pairs(n4, 2, 6)
    A, B = assemble(g4, k4)
    I = g4.interior_faces()
    K = np.block([[A[I][:, I].toarray(), B[:, I].toarray().T], [B[:, I].toarray(), np.zeros((n4 * n4, n4 * n4))]])
    x = np.linalg.lstsq(K, np.concatenate([np.zeros(I.size), g4.h ** 2 * f4.ravel()]), rcond=None)[0]
    u4, p4 = solve_direct_pinned(g4, k4, f4)
    np.testing.assert_allclose(u4[I], x[: I.size], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(p4, -(x[I.size:] - x[I.size:].mean()), rtol=1e-10, atol=1e-14)
    # channels with point sources: exact mass balance, the reduced residual
    # C^T A u at rounding level, and the bordered solve's solution (velocity
    # compared at contrast 1e4; at 1e6 the two factorisations' velocities
    # differ by conditioning, ~3e-9 here, while both residuals stay ~1e-14)
    g32 = Grid(32, 8)
    f32 = random_pairs(32, 3, 11)
    F32 = g32.h ** 2 * f32.ravel()
    C32, I32 = curl_matrix(g32), g32.interior_faces()
    for contrast, utol in ((1e4, 1e-9), (1e6, 1e-7)):
        k32 = channel_field(32, contrast, 9)
        u1, p1 = solve_direct(g32, k32, f32)
        u2, p2 = solve_direct_pinned(g32, k32, f32)
        A32, B32 = assemble(g32, k32)
        Au = (A32 @ u2)[I32]
        assert np.abs(B32 @ u2 - F32).max() <= 1e-12 * np.abs(F32).max()
        assert np.linalg.norm(C32.T @ Au) <= 1e-12 * np.linalg.norm(abs(C32.T) @ np.abs(Au))
        assert np.linalg.norm(u2 - u1) <= utol * np.linalg.norm(u1)
        assert np.linalg.norm(p2 - p1) <= 1e-12 * np.linalg.norm(p1)
        assert abs(p2.sum()) <= 1e-12 * np.abs(p2).sum()


def test_superconvergence_second_order():
    """p = cos(pi x) cos(pi y), kappa = 1: cell-centre pressure error O(h^2)."""
    errs = []
    for n in (16, 32):
        g = Grid(n, 4)
        e = (np.arange(n) + 0.5) / n
        # cell averages of cos(pi x) over [x_i, x_i + h]
        avg = (np.sin(np.pi * (e + 0.5 / n)) - np.sin(np.pi * (e - 0.5 / n))) / (np.pi / n)
        f = 2 * np.pi ** 2 * np.outer(avg, avg)
        u, p = solve_direct(g, np.ones((n, n)), f)
        pe = np.outer(np.cos(np.pi * e), np.cos(np.pi * e))
        errs.append(np.abs(p.reshape(n, n) - (pe - pe.mean())).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


# --------------------------------------------------------------------- spectral
def test_jacobi_matches_lapack():
    rng = np.random.default_rng(8)
    for trial in range(4):
        m = [5, 12, 16, 16][trial]
        Q = np.linalg.qr(rng.standard_normal((m, m)))[0]
        if trial == 3:  # clustered / repeated eigenvalues
            lam = np.repeat(rng.uniform(0.1, 10, m // 2), 2)
        else:
            lam = rng.uniform(-3, 10, m) * 10.0 ** rng.uniform(-3, 3, m)
        S = (Q * lam) @ Q.T
        S = 0.5 * (S + S.T)
        w, V = jacobi_eigh(S)
        w_ref = np.linalg.eigh(S)[0]
        np.testing.assert_allclose(w, w_ref, rtol=1e-11, atol=1e-12 * np.abs(w_ref).max())
        np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-12)
        np.testing.assert_allclose(S @ V, V * w, atol=1e-11 * np.abs(w).max())


@pytest.fixture(scope="module")
def small_problem():
    n, b = 16, 4
    g = Grid(n, b)
    kappa = lognormal_field(n, 11, sigma=2.0)
    A, B = assemble(g, kappa)
    return g, kappa, A, B, BlockSolvers(g, A, B)


def test_snapshot_boundary_and_divergence(small_problem):
    g, kappa, A, B, blocks = small_problem
    face = coarse_faces(g)[5]
    sup, val = snapshots(g, A, B, blocks, face)
    ef, _, _ = fine_faces_on(g, face)
    full = np.zeros((g.nf, g.b))
    full[sup] = val
    np.testing.assert_array_equal(full[ef], np.eye(g.b))       # v.n_i = delta_l on E_i
    (I1, J1), (I2, J2) = face_blocks(face)
    for (I, J), sgn in (((I1, J1), 1.0), ((I2, J2), -1.0)):
        fi, fb, cells, _ = blocks.get(I, J)
        other = np.setdiff1d(fb, ef)
        assert np.abs(full[other]).max() == 0.0                # zero flux elsewhere on dK
        div = (B[cells] @ full)                                 # int_c div v
        np.testing.assert_allclose(div, sgn * g.h / g.b ** 2, rtol=1e-11)
        # Darcy law inside K: A v lies in the range of B_K^T (a discrete gradient)
        Av = (A[fi] @ full)
        BK = B[cells][:, fi].toarray()
        coef = np.linalg.lstsq(BK.T, Av, rcond=None)[0]
        assert np.abs(BK.T @ coef - Av).max() <= 1e-11 * np.abs(Av).max()


def test_spectral_problem_against_generalized_lapack(small_problem):
    g, kappa, A, B, blocks = small_problem
    for face in coarse_faces(g)[:4]:
        sup, val = snapshots(g, A, B, blocks, face)
        a, s = spectral_problem(g, A, B, 1 / kappa, face, sup, val)
        lam, c = solve_spectral(a, s, tol=50.0)
        ref = sla.eigh(np.diag(a), s, eigvals_only=True)
        np.testing.assert_allclose(lam, np.sort(ref), rtol=1e-10)
        for k in range(c.shape[1]):
            rq = (c[:, k] @ (a * c[:, k])) / (c[:, k] @ s @ c[:, k])
            assert abs(rq - lam[k]) <= 1e-10 * lam[k]


def _spectral_forms_by_quadrature(n, b, kappa, face, sup, val):
    """a and s of eq. spectral_eqn for the snapshots ``val`` (on faces
    ``sup``), integrated from the velocity fields themselves, without the
    oracle's A and B.  Each snapshot is rebuilt cell by cell as an RT0 field
    (v_x linear in x between the cell's two x-face values, v_y linear in y),
    kappa^{-1} v.w is integrated with a 3 x 3 Gauss rule (exact for these
    quadratics), and div v div w with div v = (sum of outflow values) / h,
    constant per cell, times the cell area.  s = (that sum over omega) / H
    with H = b / n, the coarse block side in domain units.  a is the trace
    product sum_l kappa_e^{-1} (v.n)_l (w.n)_l over the fine faces of E, with
    kappa_e^{-1} the mean of the two adjacent cells' kappa^{-1}."""
    h = 1.0 / n
    H = b * h
    J = val.shape[1]
    nxf = (n + 1) * n
    full = np.zeros((2 * nxf, J))
    full[sup] = val
    ux = full[:nxf].reshape(n, n + 1, J)          # [j, i]: x-face at x = i h
    uy = full[nxf:].reshape(n + 1, n, J)          # [j, i]: y-face at y = j h
    kind, I, Jc = face
    blocks = ((I - 1, Jc), (I, Jc)) if kind == 0 else ((I, Jc - 1), (I, Jc))
    gx, gw = np.polynomial.legendre.leggauss(3)
    t, w = (gx + 1) / 2, gw / 2                   # nodes and weights on [0, 1]
    s = np.zeros((J, J))
    for (bI, bJ) in blocks:
        for j in range(bJ * b, (bJ + 1) * b):
            for i in range(bI * b, (bI + 1) * b):
                kinv = 1.0 / kappa[j, i]
                for tx, wx in zip(t, w):
                    for ty, wy in zip(t, w):
                        vx = ux[j, i] * (1 - tx) + ux[j, i + 1] * tx
                        vy = uy[j, i] * (1 - ty) + uy[j + 1, i] * ty
                        s += wx * wy * h * h * kinv * (np.outer(vx, vx) + np.outer(vy, vy))
                div = (ux[j, i + 1] - ux[j, i] + uy[j + 1, i] - uy[j, i]) / h
                s += h * h * np.outer(div, div)
    s /= H
    l = np.arange(b)
    if kind == 0:
        vn = ux[Jc * b + l, I * b]
        kinv_e = 0.5 * (1 / kappa[Jc * b + l, I * b - 1] + 1 / kappa[Jc * b + l, I * b])
    else:
        vn = uy[Jc * b, I * b + l]
        kinv_e = 0.5 * (1 / kappa[Jc * b - 1, I * b + l] + 1 / kappa[Jc * b, I * b + l])
    a = vn.T @ (kinv_e[:, None] * vn)
    return a, s


def test_spectral_forms_by_quadrature():
    """The scale of the spectral problem (eqs. spectral_1 and spectral_eqn of
    Section 4.2): the oracle's a and s against the same forms integrated
    from the snapshot velocity fields by quadrature.  This fixes the H^{-1}
    factor with H in domain units (reading 7), the h^{-2} of the divergence
    term, and kappa_e^{-1} as the mean of the two cells' kappa^{-1} with no
    face length (readings 5 and 6), which the selection count at kappa = 1
    constrains only within a factor of about 20."""
    for n, b, kappa in ((16, 4, lognormal_field(16, 11, sigma=2.0)),
                        (24, 8, channel_field(24, 1e4, 3))):
        g = Grid(n, b)
        A, B = assemble(g, kappa)
        blocks = BlockSolvers(g, A, B)
        faces = coarse_faces(g)
        for face in (faces[0], faces[len(faces) // 2 + 1], faces[-1]):
            sup, val = snapshots(g, A, B, blocks, face)
            a, s = spectral_problem(g, A, B, 1 / kappa, face, sup, val)
            aq, sq = _spectral_forms_by_quadrature(n, b, kappa, face, sup, val)
            np.testing.assert_allclose(a, np.diag(aq), rtol=1e-12)   # the oracle keeps a's diagonal
            assert np.abs(aq - np.diag(np.diag(aq))).max() == 0.0       # snapshots: v.n = delta_l on E
            np.testing.assert_allclose(s, sq, rtol=0, atol=1e-12 * np.abs(sq).max())


def test_kappa_one_spectrum_identical_on_all_faces():
    n, b = 16, 4
    g = Grid(n, b)
    kappa = np.ones((n, n))
    A, B = assemble(g, kappa)
    blocks = BlockSolvers(g, A, B)
    spectra = []
    for face in coarse_faces(g):
        sup, val = snapshots(g, A, B, blocks, face)
        spectra.append(solve_spectral(*spectral_problem(g, A, B, 1 / kappa, face, sup, val), 1.0)[0])
    spectra = np.array(spectra)
    np.testing.assert_allclose(spectra, np.tile(spectra[0], (len(spectra), 1)), rtol=1e-10)


def test_kappa_one_eigenfunctions_mirror_symmetric():
    """kappa = 1: the neighbourhood of a coarse face (its two blocks) is
    symmetric under reflection about the face midpoint, and the spectrum is
    simple, so each eigenfunction's coefficient vector over the face's
    snapshots (ordered along the face) is even or odd under reversal; the
    first (smallest lambda) is even and the parities alternate."""
    n, b = 16, 4
    g = Grid(n, b)
    kappa = np.ones((n, n))
    A, B = assemble(g, kappa)
    blocks = BlockSolvers(g, A, B)
    for face in coarse_faces(g):
        sup, val = snapshots(g, A, B, blocks, face)
        lam, c = solve_spectral(*spectral_problem(g, A, B, 1 / kappa, face, sup, val), 1e12)
        assert np.all(np.diff(lam) > 1e-6 * lam[-1])
        for k in range(c.shape[1]):
            v = c[:, k]
            np.testing.assert_allclose(v[::-1], (-1) ** k * v, atol=1e-12 * np.abs(v).max())


# --------------------------------------------------------------------- two-grid
def _on_divfree(s, M):
    """Eigenvalues of M A restricted to the divergence-free space (range of C)."""
    C = s.C.toarray()
    T = np.linalg.solve(C.T @ C, C.T @ M @ s.AII.toarray() @ C)
    ev = np.linalg.eigvals(T)
    assert np.abs(ev.imag).max() <= 1e-8 * np.abs(ev).max()
    return np.sort(ev.real)


def _dense(s, fn):
    return np.column_stack([fn(e) for e in np.eye(s.If.size)])


@pytest.mark.parametrize("cycle", ["multiplicative", "additive"])
def test_preconditioner_symmetric_positive_and_lanczos_cond(cycle):
    """Dense preconditioner on an 8 x 8 grid: symmetric, maps into the
    divergence-free space, and the Lanczos Cond of a converged PCG equals the
    extreme eigenvalue ratio of M A on that space."""
    n, b = 8, 4
    kappa = lognormal_field(n, 13, sigma=2.0)
    s = TwoGridSolver(n, b, kappa, tol=50.0, cycle=cycle)
    m = s.If.size
    M = np.column_stack([s.precondition(e) for e in np.eye(m)])
    assert np.abs(M - M.T).max() <= 1e-11 * np.abs(M).max()
    assert np.abs(s.BI @ M).max() <= 1e-11 * np.abs(M).max()
    C = s.C.toarray()
    T = np.linalg.solve(C.T @ C, C.T @ M @ s.AII.toarray() @ C)
    ev = np.linalg.eigvals(T)
    assert np.abs(ev.imag).max() <= 1e-8 * np.abs(ev).max()
    ev = np.sort(ev.real)
    assert ev[0] > 0
    out = s.solve(random_pairs(n, 2, 14), rtol=1e-14)
    assert abs(out["cond"] / (ev[-1] / ev[0]) - 1) < 0.02


def test_cycles_against_operator_algebra():
    """On a 12 x 12 grid with 4 x 4 blocks, as dense operators on the
    divergence-free space: the coarse correction P A is the A-orthogonal
    projection onto the coarse divergence-free space (eigenvalues 0 and 1, as
    many 1s as the coarse space's divergence-free dimension); the additive
    cycle's spectrum lies in (0, lambda_max(S A) + 1] (sum of two operators
    self-adjoint in the A inner product); and the multiplicative cycle with
    m1 = 1, m2 = 0 is S + P - P A S (residual recomputed between the two
    steps, eq. smooth then eq. coarsepre)."""
    n, b = 12, 4
    kappa = lognormal_field(n, 21, sigma=1.5)
    add = TwoGridSolver(n, b, kappa, tol=50.0, cycle="additive")
    mul = TwoGridSolver(n, b, kappa, tol=50.0, m1=1, m2=0)
    S = _dense(add, add.smoother)
    P = _dense(add, add.coarse_correction)
    A = add.AII.toarray()
    evP = _on_divfree(add, P)
    assert np.all(np.minimum(np.abs(evP), np.abs(evP - 1)) < 1e-9)
    # coarse divergence-free dimension: basis functions minus the rank of the coarse divergence
    Phi = add.Phi.toarray()
    BH = (add.PH.T @ add.BI @ add.Phi).toarray()
    dim = Phi.shape[1] - np.linalg.matrix_rank(BH)
    assert int(np.sum(evP > 0.5)) == dim
    evS = _on_divfree(add, S)
    evA = _on_divfree(add, _dense(add, add.precondition))
    assert evA[0] > 0 and evA[-1] <= evS[-1] + 1 + 1e-9
    assert evA[-1] >= max(evS[-1], 1.0) - 1e-9
    Mm = _dense(mul, mul.precondition)
    np.testing.assert_allclose(Mm, S + P - P @ A @ S, atol=1e-10 * np.abs(Mm).max())


def test_no_oversampling_gives_a_singular_preconditioner():
    """With K_i^+ = K_i (no oversampling) the local zero-flux problems never
    touch the fine faces on the coarse grid lines, and the coarse space holds
    only a few functions per coarse face: M A has zero eigenvalues on the
    divergence-free space (the library rejects overlap 0).  One cell of
    oversampling removes them."""
    n, b = 12, 4
    kappa = lognormal_field(n, 21, sigma=1.5)
    for ov, singular in ((0, True), (1, False)):
        s = TwoGridSolver(n, b, kappa, tol=50.0, overlap=ov)
        ev = _on_divfree(s, _dense(s, s.precondition))
        assert (abs(ev[0]) < 1e-12 * ev[-1]) == singular, (ov, ev[0])


def test_model1_kappa_one_paper_pin():
    """Section 6, Model 1 with k_1 = 1 (kappa == 1 needs no figure): 100 x 100
    fine, 10 x 10 coarse, eta = 0.2, K_i^+ = K_i + 2, m1 = m2 = 1, tolerance 10.
    The paper prints Cond 3.6 and N_iter 17 for the RT0, MsFEM and GMsFEM coarse
    spaces and Dim 282 (one basis per coarse face).  The source is not stated
    (quarter five-spot used), so N_iter is checked only loosely."""
    n, b = 100, 10
    kappa = np.ones((n, n))
    f = quarter_five_spot(n)
    for kind in ("gmsfem", "msfem", "rt0"):
        s = TwoGridSolver(n, b, kappa, tol=10.0, coarse=kind)
        if kind == "gmsfem":
            lam = np.array(s.info["lam"])
            assert lam[:, 0].max() < 10.0 <= lam[:, 1].min()
            assert set(s.info["nsel"]) == {1}
        assert s.coarse_dim == 281
        out = s.solve(f, rtol=1e-7)
        assert 3.5 <= out["cond"] <= 3.7
        assert 10 <= out["iters"] <= 20
