"""Sections 3, 5 and 6: preprocessing, two-grid preconditioner, PCG (oracle, FP64).

Test infrastructure only (see the package docstring).

All vectors of the Krylov iteration live on the interior faces of the fine
grid (the degrees of freedom of V_h^0).  PCG runs in the divergence-free
subspace ker B_h (Section 3): the search directions are divergence free, and
the residual is kept in ker B_h by the l2-orthogonal projection
P = I - B^T (B B^T)^+ B, which removes the discrete-gradient part B^T p that
b - A x would otherwise carry (that part does not decay, and at 1e-9 relative
residual its rounding pollutes (r, z)).  In exact arithmetic the iterates are
those of plain PCG on eq. reduced_fine_system.  The residual size is
||C^T r||_2 with C the discrete curl (the l2 residual of the divergence-free
problem); the iteration stops once that has dropped by the factor rtol
(Section 6 uses 1e-7).
"""

import numpy as np
import scipy.sparse as sp

from .fine import SaddleSolver, assemble, boundary_lift, curl_matrix
from .coarse import BlockSolvers, build_coarse_space, coarse_faces, rt0_interpolation


def lanczos_cond(alphas, betas):
    """Condition number estimate of the preconditioned operator from the CG
    coefficients (the Lanczos tridiagonal matrix that CG builds implicitly):
    T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j.
    The paper does not say how its "Cond" was obtained; this reading is the
    usual by-product of PCG."""
    m = len(alphas)
    if m == 0:
        return 1.0
    d = np.array([1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
                  for j in range(m)])
    e = np.array([np.sqrt(betas[j]) / alphas[j] for j in range(m - 1)])
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    w = np.linalg.eigvalsh(T)
    return float(w[-1] / w[0])


class TwoGridSolver:
    """Steps 1-4 of Section 5 for a fixed permeability field.

    Step 2 (setup): adaptive coarse space (Section 4) with the coarse matrix
    L_H = R_0 L_h R_0^T factored once; oversampled local matrices L_i^+
    factored once (direct solvers for all subdomain and coarse problems,
    Section 5).  ``coarse`` selects the comparator coarse spaces ('rt0',
    'msfem') instead of 'gmsfem'.  ``cycle`` = 'multiplicative' is the
    two-grid cycle of Section 5; 'additive' is the two-level Schwarz
    preconditioner S + P that Section 5 contrasts it with (no residual
    recomputed between the two parts; m1 and m2 unused)."""

    def __init__(self, n, b, kappa, tol=10.0, eta=0.2, overlap=2, m1=1, m2=1,
                 coarse="gmsfem", cap=None, profiles=None, cycle="multiplicative"):
        from .fine import Grid
        if cycle not in ("multiplicative", "additive"):
            raise ValueError("cycle must be 'multiplicative' or 'additive'")
        self.g = g = Grid(n, b, overlap)
        self.kappa = np.asarray(kappa, float).reshape(n, n)
        self.eta, self.m1, self.m2, self.cycle = eta, m1, m2, cycle
        self.A, self.B = assemble(g, self.kappa)
        self.If = g.interior_faces()
        self.pos = -np.ones(g.nf, dtype=np.int64)
        self.pos[self.If] = np.arange(self.If.size)
        self.AII = self.A[self.If][:, self.If].tocsr()
        self.BI = self.B[:, self.If].tocsr()
        self.C = curl_matrix(g)
        BBt = (self.BI @ self.BI.T).tocsr()
        self.grad_solver = SaddleSolver(BBt, sp.csr_matrix(np.ones((1, g.ncell))))
        self.blocks = BlockSolvers(g, self.A, self.B)
        # coarse cell prolongation P_H (fine cells x coarse cells)
        jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        coarse_of = ((jj // b) * g.nc + (ii // b)).ravel()
        self.PH = sp.csr_matrix((np.ones(n * n), (np.arange(n * n), coarse_of)),
                                shape=(n * n, g.nc ** 2))
        # Step 2: coarse space and coarse matrix L_H (eq. coarsepre)
        self.Phi, self.info = build_coarse_space(g, self.A, self.B, self.kappa, coarse, tol, cap,
                                                 self.blocks, profiles)
        self.coarse_solver = self._galerkin(self.Phi)
        # oversampled local matrices L_i^+ (eq. smooth)
        self.patches = []
        for J in range(g.nc):
            for I in range(g.nc):
                fi, _, cells = g.rect(*g.patch_rect(I, J))
                self.patches.append((self.pos[fi], SaddleSolver(self.A[fi][:, fi],
                                                                self.B[cells][:, fi])))
        # coarse RT0 space used by the preprocessing (Section 3)
        faces = coarse_faces(g)
        r, v, c = [], [], []
        for k, face in enumerate(faces):
            sup, val = rt0_interpolation(g, face)
            r.append(self.pos[sup]); v.append(val); c.append(np.full(sup.size, k))
        self.PiRT = sp.csc_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))),
                                  shape=(self.If.size, len(faces)))
        self.rt0_solver = self._galerkin(self.PiRT)

    # ------------------------------------------------------------------
    def _galerkin(self, Phi):
        """Factor L_H = R_0 [[A_h, B_h^T], [B_h, 0]] R_0^T with R_0^T = diag(Phi, P_H)."""
        AH = (Phi.T @ self.AII @ Phi).toarray()
        BH = (self.PH.T @ self.BI @ Phi).toarray()
        return SaddleSolver(sp.csr_matrix(0.5 * (AH + AH.T)), sp.csr_matrix(BH))

    @property
    def coarse_dim(self):
        """Dim as counted in the paper's tables: velocity basis + coarse cells + 1."""
        return self.Phi.shape[1] + self.g.nc ** 2 + 1

    # Section 5 ---------------------------------------------------------
    def smoother(self, r):
        """S r = sum_i eta R_i^{+T} L_i^{+-1} R_i^+ [r; 0] (eq. smooth), velocity part."""
        z = np.zeros_like(r)
        for idx, sol in self.patches:
            v, _, _ = sol.solve(r[idx], np.zeros(sol.k))
            z[idx] += self.eta * v
        return z

    def coarse_correction(self, r):
        """P r = R_H^T L_H^{-1} R_H [r; 0] (eq. coarsepre), velocity part."""
        c = self.Phi.T @ r
        d, _, _ = self.coarse_solver.solve(c, np.zeros(self.g.nc ** 2))
        return self.Phi @ d

    def precondition(self, r):
        """Two-grid cycle: m1 smoothing steps, one coarse step, m2 smoothing
        steps, recomputing the residual after every step (Section 5).  The
        additive cycle applies both parts to r itself: S r + P r."""
        if self.cycle == "additive":
            return self.smoother(r) + self.coarse_correction(r)
        x = np.zeros_like(r)
        for _ in range(self.m1):
            x = x + self.smoother(r - self.AII @ x)
        x = x + self.coarse_correction(r - self.AII @ x)
        for _ in range(self.m2):
            x = x + self.smoother(r - self.AII @ x)
        return x

    def project(self, r):
        """l2-orthogonal projection onto ker B_h (removes B^T y, B B^T y = B r)."""
        y, _, _ = self.grad_solver.solve(self.BI @ r, np.zeros(1))
        return r - self.BI.T @ y

    def residual_norm(self, r):
        return float(np.linalg.norm(self.C.T @ r))

    def pcg(self, bvec, rtol=1e-7, maxiter=2000):
        """Preconditioned CG from a zero initial guess (Section 6) on the
        reduced system; stops when ||C^T r|| <= rtol ||C^T r_0||."""
        x = np.zeros_like(bvec)
        r = self.project(bvec)
        res0 = self.residual_norm(r)
        hist, alphas, betas = [1.0], [], []
        if res0 == 0.0:
            return x, 0, hist, alphas, betas
        z = self.precondition(r)
        p = z.copy()
        rz = r @ z
        it = 0
        for it in range(1, maxiter + 1):
            q = self.project(self.AII @ p)
            pq = p @ q
            if not pq > 0:
                raise FloatingPointError("PCG breakdown: p^T A p <= 0")
            alpha = rz / pq
            x += alpha * p
            r -= alpha * q
            alphas.append(alpha)
            hist.append(self.residual_norm(r) / res0)
            if hist[-1] <= rtol:
                break
            z = self.precondition(r)
            rz_new = r @ z
            beta = rz_new / rz
            betas.append(beta)
            p = z + beta * p
            rz = rz_new
        return x, it, hist, alphas, betas

    # Section 3 ---------------------------------------------------------
    def preprocess(self, Fp, gvel):
        """vbar_h with B_h vbar_h = F_h: coarse RT0 solve, then one zero-flux
        Neumann problem per coarse block with data (g - A vbar_H, F - B vbar_H)
        (eq. subproblem).  Fp is the divergence data after lifting the
        boundary flux, gvel the matching velocity data (zero for no flow)."""
        g = self.g
        cH, _, _ = self.rt0_solver.solve(self.PiRT.T @ gvel, self.PH.T @ Fp)
        vH = self.PiRT @ cH
        rv = gvel - self.AII @ vH
        rs = Fp - self.BI @ vH
        vbar = vH.copy()
        for J in range(g.nc):
            for I in range(g.nc):
                fi, _, cells, sol = self.blocks.get(I, J)
                v, _, _ = sol.solve(rv[self.pos[fi]], rs[cells])
                vbar[self.pos[fi]] += v
        return vbar

    def pressure(self, u_full):
        """Least-squares pressure from A u - B^T p = 0 on interior faces:
        (B B^T) p = B (A u), with sum(p) = 0 (physical sign)."""
        rhs = self.BI @ (self.A @ u_full)[self.If]
        BBt = (self.BI @ self.BI.T).tocsr()
        one = sp.csr_matrix(np.ones((BBt.shape[0], 1)))
        K = sp.bmat([[BBt, one], [one.T, None]], format="csc")
        from scipy.sparse.linalg import spsolve
        sol = spsolve(K, np.concatenate([rhs, [0.0]]))
        return sol[:-1]

    def solve(self, f, bflux=None, rtol=1e-7, maxiter=2000):
        """Steps 1, 3 and 4: preprocessing, PCG on the reduced system, and
        v_h = vbar_h + vtilde_h; then the pressure.  Returns a dict."""
        g = self.g
        uB = boundary_lift(g, bflux)
        F = g.h ** 2 * np.asarray(f, float).ravel()
        Fp = F - self.B @ uB
        if abs(Fp.sum()) > 1e-12 * max(1.0, np.abs(F).sum() + g.h * np.abs(uB).sum()):
            raise ValueError("incompatible source: sum(F) != net boundary outflow")
        gvel = -(self.A @ uB)[self.If]
        vbar = self.preprocess(Fp, gvel)
        bvec = gvel - self.AII @ vbar
        vt, iters, hist, alphas, betas = self.pcg(bvec, rtol, maxiter)
        u = uB.copy()
        u[self.If] = vbar + vt
        p = self.pressure(u)
        return {"u": u, "p": p, "iters": iters, "hist": hist, "vbar": vbar,
                "cond": lanczos_cond(alphas, betas), "alphas": alphas, "betas": betas}
