"""Section 2: the two-scale grid and the RT0/P0 fine system (oracle, FP64).

Test infrastructure only (see the package docstring).

Grid conventions (oracle's own):
  * fine cells (i, j), i, j in [0, n): [i h, (i+1) h] x [j h, (j+1) h], h = 1/n,
    flat index j*n + i (x fastest);
  * x-faces (normal +x) (i, j), i in [0, n], j in [0, n): flat j*(n+1) + i;
  * y-faces (normal +y) (i, j), i in [0, n), j in [0, n]: flat nxf + j*n + i;
  * nodes (i, j), i, j in [0, n]: flat j*(n+1) + i.
The face unknown is the normal velocity value (RT0 degree of freedom with
unit value on its face), so the flux through a face is h times the unknown.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class Grid:
    """Fine grid T_h of n x n square cells refined from the coarse grid T_H of
    (n/b) x (n/b) blocks K_i (Section 2, Fig. 1).  ``overlap`` is the number
    of fine cells by which an oversampled block K_i^+ extends K_i on each side
    (Section 6: K_i^+ = K_i + 2)."""

    def __init__(self, n, b, overlap=2):
        if n % b:
            raise ValueError("the block size b must divide n")
        self.n, self.b, self.ov = int(n), int(b), int(overlap)
        self.nc = self.n // self.b
        self.h = 1.0 / self.n
        self.H = self.b * self.h
        self.nxf = (self.n + 1) * self.n
        self.nyf = self.n * (self.n + 1)
        self.nf = self.nxf + self.nyf
        self.ncell = self.n * self.n

    # flat indices --------------------------------------------------------
    def xface(self, i, j):
        return np.asarray(j) * (self.n + 1) + np.asarray(i)

    def yface(self, i, j):
        return self.nxf + np.asarray(j) * self.n + np.asarray(i)

    def cell(self, i, j):
        return np.asarray(j) * self.n + np.asarray(i)

    def node(self, i, j):
        return np.asarray(j) * (self.n + 1) + np.asarray(i)

    # index sets ------------------------------------------------------------
    def rect(self, x0, x1, y0, y1):
        """Faces and cells of the cell rectangle [x0, x1) x [y0, y1).

        Returns (interior faces, boundary faces, cells) as flat index arrays;
        interior faces are those whose two neighbouring cells both lie in the
        rectangle, i.e. the degrees of freedom of V_h cap H_0(div, rect)."""
        jj, ii = np.meshgrid(np.arange(y0, y1), np.arange(x0 + 1, x1), indexing="ij")
        xin = self.xface(ii, jj).ravel()
        jj, ii = np.meshgrid(np.arange(y0 + 1, y1), np.arange(x0, x1), indexing="ij")
        yin = self.yface(ii, jj).ravel()
        js = np.arange(y0, y1)
        is_ = np.arange(x0, x1)
        xbd = np.concatenate([self.xface(x0, js), self.xface(x1, js)])
        ybd = np.concatenate([self.yface(is_, y0), self.yface(is_, y1)])
        jj, ii = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
        cells = self.cell(ii, jj).ravel()
        return (np.sort(np.concatenate([xin, yin])),
                np.sort(np.concatenate([xbd, ybd])), cells)

    def interior_faces(self):
        """Degrees of freedom of V_h^0 (faces not on the boundary of D)."""
        return self.rect(0, self.n, 0, self.n)[0]

    def block_rect(self, I, J):
        b = self.b
        return I * b, (I + 1) * b, J * b, (J + 1) * b

    def patch_rect(self, I, J):
        """Oversampled block K_i^+ of block (I, J), clipped at the boundary of D."""
        b, ov, n = self.b, self.ov, self.n
        return (max(0, I * b - ov), min(n, (I + 1) * b + ov),
                max(0, J * b - ov), min(n, (J + 1) * b + ov))


def assemble(g, kappa):
    """RT0/P0 matrices of eq. fine_system on all faces (boundary faces included).

    A[f, e] = int kappa^{-1} phi_f . phi_e  (exact integration, cell by cell),
    B[c, f] = int_c div phi_f               (= +h / -h for outflow / inflow).
    kappa is an (n, n) array indexed [j, i] (x fastest when flattened)."""
    n, h = g.n, g.h
    kinv = 1.0 / np.asarray(kappa, dtype=np.float64).reshape(n, n)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    c = g.cell(ii, jj).ravel()
    k = kinv.ravel()
    fl, fr = g.xface(ii, jj).ravel(), g.xface(ii + 1, jj).ravel()
    fb, ft = g.yface(ii, jj).ravel(), g.yface(ii, jj + 1).ravel()
    # On a square cell the two x-basis functions are (x_{i+1}-x)/h and
    # (x-x_i)/h; their L2 products are h^2/3 (same) and h^2/6 (other).
    d, o = h * h / 3.0 * k, h * h / 6.0 * k
    rows = np.concatenate([fl, fr, fl, fr, fb, ft, fb, ft])
    cols = np.concatenate([fl, fr, fr, fl, fb, ft, ft, fb])
    vals = np.concatenate([d, d, o, o, d, d, o, o])
    A = sp.csr_matrix((vals, (rows, cols)), shape=(g.nf, g.nf))
    one = np.full(n * n, h)
    B = sp.csr_matrix((np.concatenate([one, -one, one, -one]),
                       (np.concatenate([c, c, c, c]), np.concatenate([fr, fl, ft, fb]))),
                      shape=(g.ncell, g.nf))
    return A, B


def boundary_lift(g, bflux):
    """Face vector carrying the prescribed boundary normal velocities.

    bflux (length 4n, or None for no flow) holds the OUTWARD normal velocity
    on the left (j = 0..n-1), right (j), bottom (i = 0..n-1) and top (i)
    boundary faces, in that order.  The paper's problem is the homogeneous
    case v.n = 0 (Section 2)."""
    u = np.zeros(g.nf)
    if bflux is None:
        return u
    bf = np.asarray(bflux, dtype=np.float64).reshape(4, g.n)
    k = np.arange(g.n)
    u[g.xface(0, k)] = -bf[0]
    u[g.xface(g.n, k)] = bf[1]
    u[g.yface(k, 0)] = -bf[2]
    u[g.yface(k, g.n)] = bf[3]
    return u


class SaddleSolver:
    """Direct solver for a zero-flux (pure Neumann) saddle-point block
    [[A_ff, B_cf^T], [B_cf, 0]] on the given faces and cells, as used for the
    local matrices L_i, L_i^+ and L_H of Section 2 and the direct solvers of
    Section 5.  The pressure is fixed by one extra Lagrange row sum(p) = 0;
    the multiplier of that row is returned so that callers can check that the
    divergence data were compatible (it is then zero)."""

    def __init__(self, A, Bm, check=True):
        A = sp.csr_matrix(A)
        Bm = sp.csr_matrix(Bm)
        self.m, self.k = A.shape[0], Bm.shape[0]
        one = sp.csr_matrix(np.ones((self.k, 1)))
        self.K = sp.bmat([[A, Bm.T, None], [Bm, None, one], [None, one.T, None]], format="csc")
        self.lu = spla.splu(self.K)

    def solve(self, gvel, sdiv, refine=0):
        """refine: steps of iterative refinement (residual of the bordered
        system in FP64, correction from the same LU factors)."""
        rhs = np.concatenate([np.asarray(gvel, float), np.asarray(sdiv, float), [0.0]])
        x = self.lu.solve(rhs)
        for _ in range(refine):
            x = x + self.lu.solve(rhs - self.K @ x)
        return x[: self.m], x[self.m: self.m + self.k], x[-1]


def solve_direct(g, kappa, f, bflux=None):
    """Exact discrete solution of eq. fine_system with a sparse direct solver.

    f is the cell-average source density (F_c = h^2 f_c).  Returns the full
    face vector u (boundary values included) and the PHYSICAL pressure
    p = -p_paper (the paper's matrix carries +B^T, so its p has the opposite
    sign of the weak form's), normalised to sum(p) = 0.  The unknown count
    is interior faces + cells + 1, the DOF convention of Section 6.

    The LU solution takes one step of iterative refinement in FP64 (same
    factors).  At contrast 1e6 the unrefined solution's velocities carry a
    relative l2 error of a few 1e-8 (the channels' velocities are weighted by
    kappa^{-1} ~ 1e-6 in A, so its energy-norm error stays ~1e-10); the
    refined one agrees with the converged FP64 PCG to ~2e-9."""
    A, B = assemble(g, kappa)
    uB = boundary_lift(g, bflux)
    F = g.h ** 2 * np.asarray(f, dtype=np.float64).ravel()
    I = g.interior_faces()
    s = F - B @ uB
    if abs(s.sum()) > 1e-12 * max(1.0, np.abs(F).sum() + g.h * np.abs(uB).sum()):
        raise ValueError("incompatible source: sum(F) != net boundary outflow")
    sol = SaddleSolver(A[I][:, I], B[:, I])
    v, p_paper, mu = sol.solve(-(A @ uB)[I], s, refine=1)
    u = uB.copy()
    u[I] = v
    return u, -p_paper


def solve_direct_pinned(g, kappa, f, bflux=None):
    """The same exact discrete solution as solve_direct (eq. fine_system,
    physical pressure with sum(p) = 0), for large grids.  The pressure's free
    constant (pure Neumann problem, Section 2) is fixed during the
    factorisation by removing cell 0's row of B (its pressure is 0), and the
    pressure is shifted to zero mean afterwards.  This leaves the saddle matrix
    without the dense Lagrange row of solve_direct, so the sparse LU stays
    sparse (seconds at 256 x 256 instead of minutes).  The dropped row is
    implied by the others, since sum(F) equals the net boundary outflow.
    One step of FP64 iterative refinement follows, as in solve_direct."""
    A, B = assemble(g, kappa)
    uB = boundary_lift(g, bflux)
    F = g.h ** 2 * np.asarray(f, dtype=np.float64).ravel()
    I = g.interior_faces()
    s = F - B @ uB
    if abs(s.sum()) > 1e-12 * max(1.0, np.abs(F).sum() + g.h * np.abs(uB).sum()):
        raise ValueError("incompatible source: sum(F) != net boundary outflow")
    AI, BI = A[I][:, I], B[:, I][1:]
    K = sp.bmat([[AI, BI.T], [BI, None]], format="csc")
    lu = spla.splu(K)
    rhs = np.concatenate([-(A @ uB)[I], s[1:]])
    x = lu.solve(rhs)
    x = x + lu.solve(rhs - K @ x)
    u = uB.copy()
    u[I] = x[: I.size]
    p = -np.concatenate([[0.0], x[I.size:]])
    return u, p - p.mean()


def split_faces(g, u):
    """Full face vector -> (ux (n, n+1) indexed [j, i], uy (n+1, n) indexed [j, i])."""
    return u[: g.nxf].reshape(g.n, g.n + 1), u[g.nxf:].reshape(g.n + 1, g.n)


def curl_matrix(g):
    """Discrete curl C: stream function on interior nodes -> normal velocity
    on interior faces, u_x(i, j) = (psi(i, j+1) - psi(i, j)) / h,
    u_y(i, j) = -(psi(i+1, j) - psi(i, j)) / h.  B C = 0 exactly; it is used
    only to measure the residual of the reduced (divergence-free) system."""
    n, h = g.n, g.h
    rows, cols, vals = [], [], []
    jj, ii = np.meshgrid(np.arange(n), np.arange(n + 1), indexing="ij")
    f = g.xface(ii, jj).ravel()
    rows += [f, f]
    cols += [g.node(ii, jj + 1).ravel(), g.node(ii, jj).ravel()]
    vals += [np.full(f.size, 1.0 / h), np.full(f.size, -1.0 / h)]
    jj, ii = np.meshgrid(np.arange(n + 1), np.arange(n), indexing="ij")
    f = g.yface(ii, jj).ravel()
    rows += [f, f]
    cols += [g.node(ii + 1, jj).ravel(), g.node(ii, jj).ravel()]
    vals += [np.full(f.size, -1.0 / h), np.full(f.size, 1.0 / h)]
    C = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(g.nf, (n + 1) ** 2))
    jj, ii = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
    inner_nodes = g.node(ii, jj).ravel()
    return C[g.interior_faces()][:, inner_nodes]
