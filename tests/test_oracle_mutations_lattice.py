"""Plausible mistakes planted in the lattice and mixed-state parts of the oracle each make one of
their pins fail (no GPU); see test_oracle_mutations.py for the solver's own oracle."""

import importlib.util
import os

import numpy as np
import pytest

import oracle.ed_oracle as OE
import oracle.lattice_oracle as LO

HERE = os.path.dirname(os.path.abspath(__file__))


def _load(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(HERE, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PL = _load("test_lattice_oracle_pins")
PM = _load("test_mixed_oracle_pins")


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_mixed_hopping_phase_with_the_wrong_sign(monkeypatch):
    """e^{-i k.r} instead of e^{i k.r} in the mixed representation of Sec. 2.2."""
    real = LO.mixed_hopping

    def wrong(t_c, bonds, E, kt):
        return real(t_c, bonds, E, -np.asarray(kt))
    monkeypatch.setattr(LO, "mixed_hopping", wrong)
    _fails(PL.test_mixed_hopping_worked_example)


def test_inter_cluster_term_added_instead_of_subtracted(monkeypatch):
    """G^-1 = G_c^-1 + V instead of G_c^-1 - V (Eq. CPT1)."""
    real = LO.cpt_green

    def wrong(Gc, V, Gamma=None):
        return real(Gc, -np.asarray(V), Gamma)
    monkeypatch.setattr(LO, "cpt_green", wrong)
    _fails(PL.test_cpt_exact_at_u0, 2, 1, 0.0)


def test_hybridization_with_one_factor_of_theta(monkeypatch):
    """theta_{mu a} in place of theta_{mu a} theta_{nu a} (a dropped factor)."""
    def wrong(theta, eps, z):
        theta = np.asarray(theta, dtype=float)
        z = np.asarray(z, dtype=complex).ravel()
        g = 1.0 / (z[:, None] - np.asarray(eps)[None, :])
        return np.einsum("ma,na,ka->kmn", theta, np.ones_like(theta), g)
    monkeypatch.setattr(LO, "hybridization", wrong)
    _fails(PL.test_hybridization_schur_complement)


def test_superlattice_sum_without_its_normalization(monkeypatch):
    """(L/N) sum over k~ taken as the plain sum."""
    real = LO.cpt_green
    monkeypatch.setattr(LO, "superlattice_average", lambda Gc, V, Gamma=None: real(Gc, V, Gamma).sum(axis=0))
    _fails(PL.test_superlattice_average_real_space, 4, 1, (6,))


def test_self_energy_with_the_inverse_added(monkeypatch):
    """Sigma = z - h_c - Gamma + G_c^-1 (a sign error)."""
    def wrong(Gc, z, h_c, Gamma=None):
        z = np.asarray(z, dtype=complex).ravel()
        S = z[:, None, None] * np.eye(h_c.shape[0]) - h_c[None] + np.linalg.inv(Gc)
        return S - Gamma if Gamma is not None else S
    monkeypatch.setattr(LO, "self_energy", wrong)
    _fails(PL.test_self_energy_vanishes_at_u0)


def test_excited_states_measured_from_the_ground_energy(monkeypatch):
    """Every state's Green function built with E_0 as its reference energy instead of E_s."""
    real = OE.green_exact

    def wrong(model, n_up, n_dn, z, spin=0, orbitals=None, dense_limit=6000, state=None):
        if state is not None:
            E0 = OE.low_states(OE.sector_hamiltonian(model, n_up, n_dn), 1)[0][0]
            state = (E0, state[1])
        return real(model, n_up, n_dn, z, spin, orbitals, dense_limit, state)
    monkeypatch.setattr(OE, "green_exact", wrong)
    _fails(PM.test_free_fermion_mixture_at_any_temperature_is_the_resolvent)


def test_boltzmann_weights_not_normalized(monkeypatch):
    def wrong(E, T, degenerate_tol=1e-9):
        E = np.asarray(E, dtype=float)
        return np.exp(-(E - E[0]) / T) if T > 0 else (E - E[0] <= degenerate_tol).astype(float)
    monkeypatch.setattr(OE, "mixed_weights", wrong)
    _fails(PM.test_mixed_green_of_degenerate_free_states_is_the_resolvent)
