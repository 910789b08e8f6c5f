"""Plausible mistakes planted in the CPU oracle each make one of its pins fail (no GPU).

Each test replaces one piece of the oracle with a wrong variant (monkeypatch, undone after the
test) and runs a pin from test_oracle_pins.py, which must then raise.  This shows that the pins
constrain the oracle: a dropped term, a wrong sign or a wrong factor does not pass them."""

import importlib.util
import os

import numpy as np
import pytest

import oracle as O
import oracle.ed_oracle as OE

_spec = importlib.util.spec_from_file_location(
    "oracle_pins", os.path.join(os.path.dirname(__file__), "test_oracle_pins.py"))
P = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(P)


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_sign_rule_counting_an_endpoint(monkeypatch):
    """(-1)^M_ab must count the occupied orbitals strictly between a and b."""
    def wrong(a, b):
        lo, hi = min(a, b), max(a, b)
        return ((1 << (hi + 1)) - 1) ^ ((1 << (lo + 1)) - 1)
    monkeypatch.setattr(OE, "_between_mask", wrong)
    _fails(P.test_factorized_matches_jordan_wigner, 2, 3, 1, 2, 2)
    _fails(P.test_worked_sign_example)


def test_chemical_potential_with_the_wrong_sign(monkeypatch):
    real = OE.one_body_matrix

    def wrong(t, mu, eps=None, theta=None):
        return real(t, -mu, eps, theta)
    monkeypatch.setattr(OE, "one_body_matrix", wrong)
    _fails(P.test_two_site_closed_form, -1.0, 8.0, 4.0)


def test_hole_fraction_with_the_electron_sign(monkeypatch):
    real = OE.cf_green

    def wrong(a, bsq, z, E0, kind):
        return real(a, bsq, z, E0, "e")
    monkeypatch.setattr(OE, "cf_green", wrong)
    _fails(P.test_one_site_atomic_green, 1, 0, 5.0, 1.5, "-mu")


def test_off_diagonal_combination_without_one_half(monkeypatch):
    real = O.green_cf

    def wrong(*args, **kw):
        G, coeffs = real(*args, **kw)
        p = G.shape[1]
        off = ~np.eye(p, dtype=bool)
        G = G.copy()
        G[:, off] *= 2.0  # (G+ - G_ii - G_jj) instead of half of it
        return G, coeffs
    monkeypatch.setattr(O, "green_cf", wrong)
    _fails(P.test_green_sum_rules_and_methods, 42, 4, 2, 3, 3)


def test_dropped_hybridization(monkeypatch):
    real = OE.one_body_matrix

    def wrong(t, mu, eps=None, theta=None):
        return real(t, mu, eps, None if theta is None else np.zeros_like(np.asarray(theta, dtype=float)))
    monkeypatch.setattr(OE, "one_body_matrix", wrong)
    _fails(P.test_site_bath_pair_closed_form, 1.0, -0.5, 0.7)


def test_jordan_wigner_string_dropped(monkeypatch):
    """Every mode anticommutes past the occupied modes before it.  (Counting the modes after it
    instead is the reversed ordering, an equally valid convention, which the pins accept.)"""
    def wrong(ops, state):
        for kind, m in reversed(ops):
            occ = (state >> m) & 1
            if kind == "+":
                if occ:
                    return 0, None
                state |= 1 << m
            else:
                if not occ:
                    return 0, None
                state &= ~(1 << m)
        return 1, state
    monkeypatch.setattr(OE, "_jw_apply", wrong)
    _fails(P.test_factorized_matches_jordan_wigner, 2, 3, 1, 2, 2)
