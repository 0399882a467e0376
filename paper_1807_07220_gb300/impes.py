"""Two-phase flow by IMPES (Section 6.2) on the library's solver.

Each step: the pressure equation with permeability kappa * lambda(s^n)
(tg_total_mobility, then tg_update_kappa on the existing handle), a solve
warm-started from the previous velocity (tg_solve_warm), and one explicit
upstream-weighted saturation step (tg_transport_step).  This module only
sequences the library's calls; every step runs in its kernels.
"""

import time

from . import tgms

COARSE_MODES = {"frozen": 0, "rebuild": 1, "frozen_full": 2}


class Impes:
    """kappa, f: (n, n) torch float64 CUDA tensors (absolute permeability,
    cell source densities: f > 0 injects water, f < 0 produces).  coarse:
    'frozen' keeps the coarse basis of the first setup (the paper's choice)
    and updates the coarse inverses by low-rank corrections; 'frozen_full'
    keeps the basis and recomputes the inverses in full; 'rebuild' rebuilds
    the basis every step by the handle's method (exact spectral problems, or
    the learned basis with coarse_space='learned')."""

    def __init__(self, kappa, f, b, eig_tol=10.0, s0=None, mu_w=1.0, mu_o=5.0, cfl=0.5, rtol=1e-8,
                 coarse="frozen", **solver_opts):
        import torch
        self.torch = torch
        self.n = kappa.shape[0]
        self.kappa = kappa.contiguous()
        self.f = f.contiguous()
        self.mu_w, self.mu_o, self.cfl, self.rtol = mu_w, mu_o, cfl, rtol
        self.coarse = COARSE_MODES[coarse]
        self.s = torch.zeros_like(self.kappa) if s0 is None else s0.clone().contiguous()
        self.s_next = torch.empty_like(self.s)
        self.keff = torch.empty_like(self.kappa)
        self.stream = torch.cuda.current_stream().cuda_stream
        tgms.tg_total_mobility(self.kappa, self.s, self.n, mu_w, mu_o, self.keff, self.stream)
        self.solver = tgms.Solver(self.keff, b, eig_tol, **solver_opts)
        self.ux_prev = None
        self.t = 0.0
        self.steps = 0
        self.history = []    # per step: (dt, PCG iterations, update ms, solve ms, transport ms, patches refactored,
                             #  rank of the coarse-inverse update (-1 = full), snapshot solves of the
                             #  current coarse space, its faces that fell back to the exact problem)

    def step(self):
        tg, torch = tgms, self.torch
        t0 = time.perf_counter()
        if self.steps > 0:
            tg.tg_total_mobility(self.kappa, self.s, self.n, self.mu_w, self.mu_o, self.keff, self.stream)
            tg.tg_update_kappa(self.solver.h, self.keff, self.coarse)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        it, rep = self.solver.solve(self.f, rtol=self.rtol, ux0=self.ux_prev)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        dt = tg.tg_transport_step(self.s, self.solver.ux, self.solver.uy, self.f, self.n, self.cfl, self.mu_w,
                                  self.mu_o, self.s_next, stream=self.stream)
        t3 = time.perf_counter()
        self.s, self.s_next = self.s_next, self.s
        self.ux_prev = self.solver.ux.clone()
        self.t += dt
        self.steps += 1
        self.history.append((dt, it, 1e3 * (t1 - t0), 1e3 * (t2 - t1), 1e3 * (t3 - t2), rep.refactored_patches,
                             rep.update_rank[0], rep.snapshot_solves, rep.fallback_faces))
        return dt, it

    def close(self):
        self.solver.close()
