"""Two-phase flow by IMPES (Section 6.2), oracle, FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Water (w) and oil (o), incompressible, porosity 1, no gravity or capillarity.
The pressure equation is the Darcy problem of Section 2 with the permeability
kappa * lambda(s), lambda the total mobility of eq. mobility; the saturation
equation (eq. satEq) is discretised by the finite-volume update of eq.
DisSatEq_Implicit with upstream weighting of the fractional flow f_w (eq.
fraction).

Readings:
  * relative permeabilities k_rw = s^2, k_ro = (1 - s)^2, viscosities given
    (the paper uses one unstated set; mu_w = 1, mu_o = 5 as in its SPE10 run);
  * the update is evaluated at s^n (explicit upwind) instead of the paper's
    backward Euler with Newton, with the time step from a CFL number:
    dt = cfl * h^2 / (F_max * sigma), F_max the largest total outflow of a
    cell (outgoing face fluxes u h plus its sink h^2 max(-f, 0)) and sigma the
    largest derivative of f_w over [0, 1] (the fastest saturation wave);
  * sources: f > 0 injects water, f < 0 produces fluid at the cell's
    fractional flow (the q+ and f_w(s_i) q- terms); a boundary face with
    inward flux injects water, one with outward flux carries f_w of its cell;
  * porosity 1, cell volume h^2.
"""

import numpy as np


def total_mobility(s, mu_w=1.0, mu_o=5.0):
    """lambda(s) = k_rw / mu_w + k_ro / mu_o (eq. mobility)."""
    s = np.asarray(s, float)
    return s * s / mu_w + (1.0 - s) * (1.0 - s) / mu_o


def frac_flow(s, mu_w=1.0, mu_o=5.0):
    """f_w(s) = (k_rw / mu_w) / lambda(s) (eq. fraction)."""
    s = np.asarray(s, float)
    return (s * s / mu_w) / total_mobility(s, mu_w, mu_o)


def frac_flow_slope(s, mu_w=1.0, mu_o=5.0):
    """df_w/ds = 2 s (1 - s) / (mu_w mu_o lambda(s)^2)."""
    s = np.asarray(s, float)
    lam = total_mobility(s, mu_w, mu_o)
    return 2.0 * s * (1.0 - s) / (mu_w * mu_o * lam * lam)


def max_slope(mu_w=1.0, mu_o=5.0, samples=20001):
    """sigma = max of df_w/ds over samples equally spaced points of [0, 1]."""
    s = np.arange(samples) / (samples - 1.0)
    return float(np.max(frac_flow_slope(s, mu_w, mu_o)))


def transport_step(n, s, ux, uy, f, cfl=0.5, mu_w=1.0, mu_o=5.0, dt=None):
    """One explicit upwind step of eq. DisSatEq_Implicit.

    s: (n, n) [j, i] cell saturations; ux (n, n+1), uy (n+1, n) normal
    velocities (+x / +y), boundary faces included; f (n, n) cell source
    densities.  Returns (s_new, dt)."""
    h = 1.0 / n
    s = np.asarray(s, float)
    ux = np.asarray(ux, float)
    uy = np.asarray(uy, float)
    f = np.asarray(f, float)
    fw = frac_flow(s, mu_w, mu_o)
    # total outflow of each cell: outgoing face fluxes plus the sink
    out = (np.maximum(ux[:, 1:], 0.0) + np.maximum(-ux[:, :-1], 0.0) +
           np.maximum(uy[1:, :], 0.0) + np.maximum(-uy[:-1, :], 0.0)) * h + h * h * np.maximum(-f, 0.0)
    if dt is None:
        fmax = float(out.max())
        dt = cfl * h * h / (fmax * max_slope(mu_w, mu_o)) if fmax > 0 else 0.0
    # upstream fractional flow on every face: the cell the flow leaves; at the
    # boundary, inward flow is water (1) and outward flow carries the cell's f_w
    one_col = np.ones((n, 1))
    left = np.hstack([one_col, fw])           # cell on the -x side of x-face i (water outside)
    right = np.hstack([fw, one_col])          # cell on the +x side
    upx = np.where(ux >= 0, left, right)
    upx[:, 0] = np.where(ux[:, 0] > 0, 1.0, fw[:, 0])
    one_row = np.ones((1, n))
    below = np.vstack([one_row, fw])
    above = np.vstack([fw, one_row])
    upy = np.where(uy >= 0, below, above)
    upy[0, :] = np.where(uy[0, :] > 0, 1.0, fw[0, :])
    wx = ux * h * upx                          # water flux through the faces, +x / +y
    wy = uy * h * upy
    net_out = (wx[:, 1:] - wx[:, :-1]) + (wy[1:, :] - wy[:-1, :])
    qplus = h * h * np.maximum(f, 0.0)
    qminus = h * h * np.minimum(f, 0.0)
    s_new = s + dt / (h * h) * (qplus - net_out + fw * qminus)
    return s_new, dt


def welge_front(mu_w=1.0, mu_o=5.0, samples=200001):
    """Buckley-Leverett shock saturation s* (tangent from (0, 0) to f_w:
    f_w(s*) / s* = f_w'(s*)) and the front speed f_w'(s*) for water
    displacing oil at s = 0, found as the maximiser of f_w(s) / s."""
    s = np.arange(1, samples) / (samples - 1.0)
    ratio = frac_flow(s, mu_w, mu_o) / s
    k = int(np.argmax(ratio))
    return float(s[k]), float(ratio[k])


def impes(g, kappa, f, s0, nsteps, cfl=0.5, mu_w=1.0, mu_o=5.0, solve=None):
    """IMPES: per step the pressure equation with kappa * lambda(s^n) (a
    direct solve unless ``solve`` is given: solve(kappa_eff) -> face vector u),
    then one transport step.  Returns the saturation history and time steps."""
    from .fine import solve_direct, split_faces
    n = g.n
    s = np.asarray(s0, float).copy()
    hist, dts = [s.copy()], []
    for _ in range(nsteps):
        keff = np.asarray(kappa, float) * total_mobility(s, mu_w, mu_o)
        u = solve(keff) if solve is not None else solve_direct(g, keff, f)[0]
        ux, uy = split_faces(g, u)
        s, dt = transport_step(n, s, ux, uy, f, cfl, mu_w, mu_o)
        hist.append(s.copy())
        dts.append(dt)
    return hist, dts
