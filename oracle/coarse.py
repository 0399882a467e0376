"""Section 4: snapshot space, local spectral problem and coarse spaces (oracle, FP64).

Test infrastructure only (see the package docstring).

Coarse faces E_i are the interior edges of the coarse grid T_H (boundary
coarse edges carry no V_h^0 degree of freedom).  Each is identified by
(kind, I, J):
  * kind 0, vertical edge x = I*H, y in [J*H, (J+1)*H], 1 <= I < nc, fixed
    normal n_i = +x, blocks K^1 = (I-1, J) and K^2 = (I, J);
  * kind 1, horizontal edge y = J*H, x in [I*H, (I+1)*H], 1 <= J < nc, fixed
    normal n_i = +y, blocks K^1 = (I, J-1) and K^2 = (I, J).
omega_i = K^1 u K^2 is the coarse neighbourhood of E_i.
"""

import numpy as np
import scipy.sparse as sp

from .fine import SaddleSolver


def coarse_faces(g):
    """All interior coarse faces as (kind, I, J): vertical ones first (J-major),
    then horizontal ones (J-major)."""
    nc = g.nc
    out = [(0, I, J) for J in range(nc) for I in range(1, nc)]
    out += [(1, I, J) for J in range(1, nc) for I in range(nc)]
    return out


def face_blocks(face):
    kind, I, J = face
    return ((I - 1, J), (I, J)) if kind == 0 else ((I, J - 1), (I, J))


def fine_faces_on(g, face):
    """Fine faces e_l (l = 0..b-1) composing E_i, and the two fine cells
    adjacent to each (the one in K^1, the one in K^2)."""
    kind, I, J = face
    b = g.b
    l = np.arange(b)
    if kind == 0:
        return (g.xface(I * b, J * b + l), g.cell(I * b - 1, J * b + l), g.cell(I * b, J * b + l))
    return (g.yface(I * b + l, J * b), g.cell(I * b + l, J * b - 1), g.cell(I * b + l, J * b))


def jacobi_eigh(S, tol=1e-15, max_sweeps=60):
    """Cyclic Jacobi eigensolver for a real symmetric matrix.

    Each rotation J(p, q) annihilates the (p, q) entry of J^T S J; the
    tangent t of the rotation angle is the smaller root of
    t^2 + 2 tau t - 1 = 0 with tau = (s_qq - s_pp) / (2 s_pq).  Sweeps stop
    when the off-diagonal Frobenius norm falls below tol times the norm of S.
    Returns (eigenvalues ascending, eigenvectors as columns)."""
    a = np.array(S, dtype=np.float64, copy=True)
    n = a.shape[0]
    v = np.eye(n)
    scale = np.linalg.norm(a)
    for _ in range(max_sweeps):
        off = np.linalg.norm(a - np.diag(np.diag(a)))
        if off <= tol * scale:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = a[p, q]
                if apq == 0.0:
                    continue
                diff = a[q, q] - a[p, p]
                if abs(diff) > 1e150 * abs(apq):
                    t = apq / diff          # tiny angle: t ~ 1/(2 tau)
                else:
                    tau = diff / (2.0 * apq)
                    t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + np.hypot(1.0, tau))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                ap, aq = a[:, p].copy(), a[:, q].copy()
                a[:, p], a[:, q] = c * ap - s * aq, s * ap + c * aq
                ap, aq = a[p, :].copy(), a[q, :].copy()
                a[p, :], a[q, :] = c * ap - s * aq, s * ap + c * aq
                a[p, q] = a[q, p] = 0.0
                vp, vq = v[:, p].copy(), v[:, q].copy()
                v[:, p], v[:, q] = c * vp - s * vq, s * vp + c * vq
    w = np.diag(a).copy()
    order = np.argsort(w, kind="stable")
    return w[order], v[:, order]


class BlockSolvers:
    """Zero-flux local saddle solvers L_i on every coarse block (Section 2),
    factored once; used for the snapshot problems (eq. snapshot_eqn) and the
    preprocessing subproblems (eq. subproblem)."""

    def __init__(self, g, A, B):
        self.g, self.A, self.B = g, A, B
        self.cache = {}

    def get(self, I, J):
        key = (I, J)
        if key not in self.cache:
            fi, fb, cells = self.g.rect(*self.g.block_rect(I, J))
            sol = SaddleSolver(self.A[fi][:, fi], self.B[cells][:, fi])
            self.cache[key] = (fi, fb, cells, sol)
        return self.cache[key]


def snapshots(g, A, B, blocks, face):
    """Snapshot functions v_l^i, l = 0..J_i-1, of eq. snapshot_eqn on omega_i.

    On each block K of omega_i the local mixed problem is solved with normal
    component delta_l^i on E_i (along n_i), zero normal flux on the rest of
    the boundary of K, and constant divergence alpha with
    int_K alpha = int_{dK} v.n (the text's "int_k" read as int_K).  Returns
    (support faces, values (support x J)), the support being the interior
    faces of K^1 and K^2 plus the fine faces of E_i."""
    ef, _, _ = fine_faces_on(g, face)
    b, h = g.b, g.h
    K1, K2 = face_blocks(face)
    parts = []
    for (I, J), outward in ((K1, +1.0), (K2, -1.0)):
        fi, fb, cells, sol = blocks.get(I, J)
        vals = np.zeros((fi.size, b))
        for l in range(b):
            vB = np.zeros(g.nf)
            vB[ef[l]] = 1.0
            # n_i is the outward normal of K^1 and the inward one of K^2, so
            # the net outflow of K is +h (K^1) or -h (K^2); int_c alpha = that / b^2.
            s = np.full(cells.size, outward * h / b ** 2) - B[cells] @ vB
            v, _, mu = sol.solve(-(A[fi] @ vB), s)
            vals[:, l] = v
        parts.append((fi, vals))
    sup = np.concatenate([parts[0][0], parts[1][0], ef])
    val = np.vstack([parts[0][1], parts[1][1], np.eye(b)])
    return sup, val


def spectral_problem(g, A, B, kinv, face, sup, val):
    """Matrices of eq. spectral_eqn in the snapshot basis.

    a(v, w) = int_{E_i} kappa^{-1} (v.n)(w.n) evaluated as the fine-face trace
    product sum_l kappa_e^{-1} (v.n)_l (w.n)_l, i.e. diagonal kappa_e^{-1} in
    the snapshot basis, with kappa_e^{-1} the mean of the two adjacent cells'
    kappa^{-1} (the trace of kappa on E_i is not defined by the text: this
    choice is parity unpinned; the scale of both forms is pinned by
    quadrature of the snapshot fields).
    Reading: the face length h is left out.  With it, kappa == 1 gives
    lambda_2 = pi/2 on every face at any resolution, so tolerance 10 would keep
    eight functions per face, against the single one (Dim 282, the RT0 count)
    that Section 6 reports for Model 1 with k_1 = 1; without it lambda_1 ~ 0.5
    and lambda_2 ~ 156 there.
    s(v, w) = H^{-1} (int_omega kappa^{-1} v.w + int_omega div v div w); the
    second integral is sum_c (B v)_c (B w)_c / h^2 for P0 divergences."""
    ef, cL, cR = fine_faces_on(g, face)
    h, H = g.h, g.H
    kflat = kinv.ravel()
    a = 0.5 * (kflat[cL] + kflat[cR])
    As = A[sup][:, sup]
    Bv = B[:, sup] @ val
    s = (val.T @ (As @ val) + (Bv.T @ Bv) / h ** 2) / H
    return a, 0.5 * (s + s.T)


def solve_spectral(a, s, tol, cap=None):
    """Generalised eigenproblem a c = lambda s c through the symmetric matrix
    D_a^{-1/2} s D_a^{-1/2} (eigenvalues mu = 1/lambda).  Returns all lambda
    ascending, and the coefficient vectors (columns) of the selected
    eigenfunctions: those with lambda < tol, at least one (a face keeps its
    first eigenfunction when none falls below tol), at most ``cap``.  Each
    selected vector is normalised to s(c, c) = 1 with non-negative total flux."""
    dm = 1.0 / np.sqrt(a)
    mu, y = jacobi_eigh(dm[:, None] * s * dm[None, :])
    lam = 1.0 / mu[::-1]
    y = y[:, ::-1]
    nsel = max(1, int(np.sum(lam < tol)))
    if cap is not None:
        nsel = min(nsel, cap)
    c = dm[:, None] * y[:, :nsel]
    for k in range(nsel):
        c[:, k] /= np.sqrt(c[:, k] @ s @ c[:, k])
        if c[:, k].sum() < 0:
            c[:, k] = -c[:, k]
    return lam, c


def rt0_interpolation(g, face):
    """Fine face values of the coarse RT0 velocity basis function of E_i
    (normal value 1 on E_i, linear across K^1 and K^2, zero normal component
    on the other coarse edges): the columns of R_H^T for V_H (Section 2)."""
    kind, I, J = face
    b = g.b
    rows, vals = [], []
    for t in range(-b + 1, b):
        w = 1.0 - abs(t) / b
        l = np.arange(b)
        if kind == 0:
            rows.append(g.xface(I * b + t, J * b + l))
        else:
            rows.append(g.yface(I * b + l, J * b + t))
        vals.append(np.full(b, w))
    return np.concatenate(rows), np.concatenate(vals)


def build_coarse_space(g, A, B, kappa, kind="gmsfem", tol=10.0, cap=None, blocks=None, profiles=None):
    """Coarse velocity space as a sparse matrix Phi (interior faces x dim).

    kind = 'gmsfem': V_ms of Section 4.2 (spectral selection with tolerance
                     tol); 'msfem': one MsFEM basis function per face
                     (eq. msfem); 'rt0': coarse RT0 interpolation;
           'learned': the spectral problem restricted to the span of
                     predicted flux profiles (``profiles``: faces x b x k,
                     see oracle.learned.ritz_select), with the exact problem
                     where the selection falls back.
    Returns (Phi, info) where info holds, per coarse face, the spectrum and
    the number of selected functions."""
    I_f = g.interior_faces()
    pos = -np.ones(g.nf, dtype=np.int64)
    pos[I_f] = np.arange(I_f.size)
    kinv = 1.0 / np.asarray(kappa, float).reshape(g.n, g.n)
    blocks = blocks or BlockSolvers(g, A, B)
    cols_r, cols_v, col = [], [], 0
    rows_c = []
    info = {"faces": coarse_faces(g), "lam": [], "nsel": [], "coef": [], "fallback": []}
    for fidx, face in enumerate(info["faces"]):
        if kind == "rt0":
            sup, v = rt0_interpolation(g, face)
            keep = pos[sup] >= 0
            cols_r.append(pos[sup[keep]])
            cols_v.append(v[keep])
            rows_c.append(np.full(keep.sum(), col))
            col += 1
            info["nsel"].append(1)
            continue
        sup, val = snapshots(g, A, B, blocks, face)
        if kind == "msfem":
            cset = np.ones((g.b, 1))
            info["nsel"].append(1)
        elif kind == "learned":
            from .learned import ritz_select
            a, s = spectral_problem(g, A, B, kinv, face, sup, val)
            lam, cset, fb = ritz_select(np.asarray(profiles[fidx], float), a, s, tol)
            if fb:
                lam, cset = solve_spectral(a, s, tol, cap)
            info["fallback"].append(fb)
            info["lam"].append(lam)
            info["nsel"].append(cset.shape[1])
            info["coef"].append(cset)
        else:
            a, s = spectral_problem(g, A, B, kinv, face, sup, val)
            lam, cset = solve_spectral(a, s, tol, cap)
            info["lam"].append(lam)
            info["nsel"].append(cset.shape[1])
            info["coef"].append(cset)
        for k in range(cset.shape[1]):
            cols_r.append(pos[sup])
            cols_v.append(val @ cset[:, k])
            rows_c.append(np.full(sup.size, col))
            col += 1
    Phi = sp.csc_matrix((np.concatenate(cols_v), (np.concatenate(cols_r), np.concatenate(rows_c))),
                        shape=(I_f.size, col))
    return Phi, info
