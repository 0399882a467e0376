"""The oracle's pins against planted mistakes (CPU only).

Each case plants one plausible mistake in the oracle (a wrong coefficient, a
flipped sign, a broken rotation, a dropped term, two indices swapped) and
checks that the pins named beside it fail: by a failed assertion, or by the
breakdown the mistake causes inside the pin.  The mistakes are planted with
monkeypatch in every module that holds the patched name, so nothing outside
this test changes.  The scale of the spectral problem (H in domain units,
the h^{-2} of its divergence term, kappa_e^{-1} as a mean, no face length)
is fixed by the quadrature pin; which trace of kappa on a fine face is meant
(reading 5) and the omitted face length (reading 6) are readings that the
quadrature restates, not facts it derives.
"""

import inspect
import textwrap

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import oracle.coarse as oc
import oracle.fine as of
import oracle.learned as ol
import oracle.twogrid as otg
import oracle.impes as oi
import tests.test_oracle_learned as lpins
import tests.test_oracle_impes as ipins
import tests.test_oracle_pins as pins
from paper_1807_07220_gb300.inputs import quarter_five_spot

MODULES = (of, oc, otg, ol, oi, oracle, pins, ipins, lpins)


def plant(monkeypatch, name, fn):
    for mod in MODULES:
        if hasattr(mod, name):
            monkeypatch.setattr(mod, name, fn)


def mass_offdiag_doubled(orig):
    """RT0 mass matrix with the h^2/6 couplings taken as h^2/3."""
    def bad(g, kappa):
        A, B = orig(g, kappa)
        D = sp.diags(A.diagonal())
        return sp.csr_matrix(D + 2.0 * (A - D)), B
    return bad


def divergence_sign_flipped(orig):
    """B with inflow and outflow exchanged."""
    def bad(g, kappa):
        A, B = orig(g, kappa)
        return A, -B
    return bad


def curl_y_sign_flipped(orig):
    """Discrete curl with u_y = +(psi(i+1, j) - psi(i, j)) / h."""
    def bad(g):
        C = orig(g).tocsr()
        d = np.where(g.interior_faces() >= g.nxf, -1.0, 1.0)
        return sp.csr_matrix(sp.diags(d) @ C)
    return bad


def jacobi_rotation_sign_flipped():
    """Jacobi rotation with s = -t c (the rotation that does not annihilate)."""
    src = inspect.getsource(oc.jacobi_eigh).replace("s = t * c", "s = -t * c")
    assert "s = -t * c" in src
    ns = {}
    exec(src, dict(oc.__dict__), ns)
    return ns["jacobi_eigh"]


def spectral_without_divergence(orig):
    """s(v, w) without its int div v div w term."""
    def bad(g, A, B, kinv, face, sup, val):
        a, s = orig(g, A, B, kinv, face, sup, val)
        Bv = B[:, sup] @ val
        s2 = s - (Bv.T @ Bv) / g.h ** 2 / g.H
        return a, 0.5 * (s2 + s2.T)
    return bad


def snapshots_swapped(orig):
    """Two snapshots of a face out of their order along the face."""
    def bad(g, A, B, blocks, face):
        sup, val = orig(g, A, B, blocks, face)
        val = np.array(val, copy=True)
        val[:, [0, 1]] = val[:, [1, 0]]
        return sup, val
    return bad


def method_with(cls, name, old, new):
    """A copy of method cls.name with the text old replaced by new."""
    src = textwrap.dedent(inspect.getsource(getattr(cls, name)))
    assert old in src
    ns = {}
    exec(src.replace(old, new), dict(otg.__dict__), ns)
    return ns[name]


def function_with(mod, name, old, new):
    src = inspect.getsource(getattr(mod, name))
    assert old in src
    ns = {}
    exec(src.replace(old, new), dict(mod.__dict__), ns)
    return ns[name]


def model1_cond():
    """The Model-1 pin's Cond check (Section 6, kappa = 1, 100 x 100 fine,
    10 x 10 coarse, GMsFEM space: the paper's Cond 3.6), with the PCG capped
    at 60 iterations so that a broken cycle fails quickly."""
    n, b = 100, 10
    s = otg.TwoGridSolver(n, b, np.ones((n, n)), tol=10.0)
    out = s.solve(quarter_five_spot(n), rtol=1e-7, maxiter=60)
    assert 3.5 <= out["cond"] <= 3.7


CLASS_CASES = {
    # the smoother without its damping eta (eq. smooth): only the paper's
    # Model-1 Cond fixes eta (3.6 at 0.2, 6.9 at 0.1; at 1 the cycle is not
    # positive and the PCG breaks down)
    "smoother_damping": ("smoother", "z[idx] += self.eta * v", "z[idx] += v", [model1_cond]),
    # the coarse step on r instead of the recomputed residual r - A x
    "cycle_residual": ("precondition", "self.coarse_correction(r - self.AII @ x)", "self.coarse_correction(r)",
                       [pins.test_cycles_against_operator_algebra]),
    # PCG with beta inverted
    "pcg_beta": ("pcg", "beta = rz_new / rz", "beta = rz / rz_new",
                 [pins.test_preconditioner_symmetric_positive_and_lanczos_cond]),
}


@pytest.mark.filterwarnings("ignore::RuntimeWarning")   # a broken cycle yields invalid values on purpose
@pytest.mark.parametrize("case", sorted(CLASS_CASES))
def test_planted_solver_mistake_fails_its_pins(monkeypatch, case):
    name, old, new, targets = CLASS_CASES[case]
    monkeypatch.setattr(otg.TwoGridSolver, name, method_with(otg.TwoGridSolver, name, old, new))
    for pin in targets:
        with pytest.raises(Exception):
            if "cycle" in inspect.signature(pin).parameters:
                pin("multiplicative")
            else:
                pin()


def test_planted_lanczos_mistake_fails_its_pin(monkeypatch):
    """The Lanczos tridiagonal with beta_j in place of sqrt(beta_j)."""
    bad = function_with(otg, "lanczos_cond", "np.sqrt(betas[j]) / alphas[j]", "betas[j] / alphas[j]")
    plant(monkeypatch, "lanczos_cond", bad)
    with pytest.raises(Exception):
        pins.test_preconditioner_symmetric_positive_and_lanczos_cond("multiplicative")


CASES = {
    "mass_offdiag": (lambda: ("assemble", mass_offdiag_doubled(of.assemble)),
                     [pins.test_layered_medium_closed_form, pins.test_superconvergence_second_order]),
    "divergence_sign": (lambda: ("assemble", divergence_sign_flipped(of.assemble)),
                        [pins.test_layered_medium_closed_form, pins.test_mass_and_divergence_by_quadrature]),
    "curl_sign": (lambda: ("curl_matrix", curl_y_sign_flipped(of.curl_matrix)),
                  [pins.test_divergence_of_curl_is_zero]),
    "jacobi_rotation": (lambda: ("jacobi_eigh", jacobi_rotation_sign_flipped()),
                        [pins.test_jacobi_matches_lapack]),
    "spectral_divergence_term": (lambda: ("spectral_problem", spectral_without_divergence(oc.spectral_problem)),
                                 [pins.test_layered_medium_closed_form]),
    "snapshot_order": (lambda: ("snapshots", snapshots_swapped(oc.snapshots)),
                       [pins.test_kappa_one_eigenfunctions_mirror_symmetric]),
    # H counted in fine cells (b) instead of domain units (b / n)
    "spectral_H_in_cells": (lambda: ("spectral_problem", function_with(oc, "spectral_problem", "h, H = g.h, g.H",
                                                                         "h, H = g.h, float(g.b)")),
                            [pins.test_spectral_forms_by_quadrature]),
    # the divergence term of s over h instead of h^2
    "spectral_div_over_h": (lambda: ("spectral_problem", function_with(oc, "spectral_problem",
                                                                         "(Bv.T @ Bv) / h ** 2", "(Bv.T @ Bv) / h")),
                            [pins.test_spectral_forms_by_quadrature]),
    # kappa_e^{-1} as the sum of the two cells' kappa^{-1}, not their mean
    "spectral_kappa_e_sum": (lambda: ("spectral_problem", function_with(oc, "spectral_problem",
                                                                          "a = 0.5 * (kflat[cL] + kflat[cR])",
                                                                          "a = kflat[cL] + kflat[cR]")),
                             [pins.test_spectral_forms_by_quadrature]),
    # the a-form with the face length h
    "spectral_face_length": (lambda: ("spectral_problem", function_with(oc, "spectral_problem",
                                                                          "a = 0.5 * (kflat[cL] + kflat[cR])",
                                                                          "a = 0.5 * h * (kflat[cL] + kflat[cR])")),
                             [pins.test_spectral_forms_by_quadrature]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_planted_mistake_fails_its_pins(monkeypatch, case):
    make, targets = CASES[case]
    name, fn = make()
    plant(monkeypatch, name, fn)
    for pin in targets:
        with pytest.raises(Exception):   # a failed assertion, or a breakdown the pin runs into
            pin()


def test_model1_cond_check_holds_unplanted():
    """Control: the capped Model-1 check passes on the oracle as it is."""
    model1_cond()


IMPES_CASES = {
    # downwind instead of upwind fractional flow on the x-faces
    "downwind": ("transport_step", "upx = np.where(ux >= 0, left, right)", "upx = np.where(ux >= 0, right, left)",
                 [ipins.test_maximum_principle_under_cfl, ipins.test_buckley_leverett_front]),
    # the CFL limit with h in place of h^2
    "cfl_scale": ("transport_step", "dt = cfl * h * h / (fmax * max_slope(mu_w, mu_o))",
                  "dt = cfl * h / (fmax * max_slope(mu_w, mu_o))", [ipins.test_maximum_principle_under_cfl]),
    # a sink producing water only, not the cell's fractional flow
    "sink_fraction": ("transport_step", "+ fw * qminus)", "+ qminus)", [ipins.test_transport_conserves_water_exactly]),
    # the viscosities exchanged in the fractional flow
    "fractional_flow": ("frac_flow", "(s * s / mu_w)", "(s * s / mu_o)", [ipins.test_mobility_closed_forms]),
}


@pytest.mark.parametrize("case", sorted(IMPES_CASES))
def test_planted_transport_mistake_fails_its_pins(monkeypatch, case):
    name, old, new, targets = IMPES_CASES[case]
    plant(monkeypatch, name, function_with(oi, name, old, new))
    for pin in targets:
        with pytest.raises(Exception):
            pin()


LEARNED_CASES = {
    # bfloat16 by truncation instead of round-to-nearest-even
    "bf16_truncation": ("bf16", "u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u = u & 0xFFFF0000",
                        [lpins.test_bf16_rounding_matches_torch]),
    # the hidden-to-hidden weight gradient transposed (same shape: hidden x hidden)
    "w2_gradient_transposed": ("backward", 'g["W2"], g["b2"] = dH2.T @ H1, dH2.sum(0)',
                               'g["W2"], g["b2"] = H1.T @ dH2, dH2.sum(0)', [lpins.test_gradient_by_central_differences]),
    # the subspace loss gradient with 2 for 4
    "loss_gradient_factor": ("subspace_loss", "dG = (4.0 / B) * (E @ G)", "dG = (2.0 / B) * (E @ G)",
                             [lpins.test_gradient_by_central_differences]),
    # Adam without the bias corrections
    "adam_bias_correction": ("adam_step", "mhat = m / (1 - beta1 ** t)", "mhat = m", [lpins.test_adam_matches_torch]),
}


@pytest.mark.parametrize("case", sorted(LEARNED_CASES))
def test_planted_network_mistake_fails_its_pins(monkeypatch, case):
    name, old, new, targets = LEARNED_CASES[case]
    plant(monkeypatch, name, function_with(ol, name, old, new))
    for pin in targets:
        with pytest.raises(Exception):
            pin()
