"""The oracle's pins against planted mistakes (CPU only).

Each case plants one plausible mistake in the oracle (a wrong coefficient, a
flipped sign, a broken rotation, a dropped term, two indices swapped) and
checks that the pins named beside it fail.  The mistakes are planted with
monkeypatch in every module that holds the patched name, so nothing outside
this test changes.  Known gaps stay documented instead of tested: the
face-length and H scalings of the spectral problem (readings 4 and 6) are
pinned only through the selection count at kappa = 1, and kappa on a coarse
face (reading 5) has no pin.
"""

import inspect

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import oracle.coarse as oc
import oracle.fine as of
import oracle.learned as ol
import oracle.twogrid as otg
import tests.test_oracle_pins as pins

MODULES = (of, oc, otg, ol, oracle, pins)


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


CASES = {
    "mass_offdiag": (lambda: ("assemble", mass_offdiag_doubled(of.assemble)),
                     [pins.test_layered_medium_closed_form, pins.test_superconvergence_second_order]),
    "divergence_sign": (lambda: ("assemble", divergence_sign_flipped(of.assemble)),
                        [pins.test_layered_medium_closed_form, pins.test_mass_and_divergence_by_quadrature]),
    "curl_sign": (lambda: ("curl_matrix", curl_y_sign_flipped(of.curl_matrix)),
                  [pins.test_divergence_of_curl_is_zero]),
    "jacobi_rotation": (lambda: ("jacobi_eigh", jacobi_rotation_sign_flipped()),
                        [pins.test_jacobi_matches_lapack, pins.test_model1_kappa_one_paper_pin]),
    "spectral_divergence_term": (lambda: ("spectral_problem", spectral_without_divergence(oc.spectral_problem)),
                                 [pins.test_model1_kappa_one_paper_pin]),
    "snapshot_order": (lambda: ("snapshots", snapshots_swapped(oc.snapshots)),
                       [pins.test_kappa_one_eigenfunctions_mirror_symmetric]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_planted_mistake_fails_its_pins(monkeypatch, case):
    make, targets = CASES[case]
    name, fn = make()
    plant(monkeypatch, name, fn)
    for pin in targets:
        with pytest.raises(AssertionError):
            pin()
