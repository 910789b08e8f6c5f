"""Pins of the oracle's low-lying states and mixed-state Green function (Sec. 4.2: several low
states when the ground state is degenerate; the Davidson_states and temperature options of the
library section, Sec. 9), against closed forms and invariances the method must satisfy."""

import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2305_18643_gb300 import workloads as W


def _model(c):
    return O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])


@pytest.mark.parametrize("t,U,mu", [(-1.0, 4.0, 0.0), (0.6, 3.0, 1.1)])
def test_dimer_full_spectrum(t, U, mu):
    """Half-filled two-site Hubbard model, N_up = N_dn = 1: the four energies are
    (U -+ sqrt(U^2 + 16 t^2)) / 2, 0 and U, each shifted by -2 mu."""
    c = W.hubbard_dimer(t, U, mu)
    E, V = O.low_states(O.sector_hamiltonian(_model(c), 1, 1), 4)
    r = math.sqrt(U * U + 16 * t * t)
    want = np.sort(np.array([(U - r) / 2, 0.0, U, (U + r) / 2])) - 2 * mu
    assert np.allclose(E, want, atol=1e-12)
    assert np.allclose(np.einsum("sud,tud->st", V, V), np.eye(4), atol=1e-12)


def test_free_fermion_low_states_by_enumeration():
    """U = 0: the many-body levels of a sector are sums of single-particle levels over occupied
    orbitals, enumerated here configuration by configuration; the k lowest agree."""
    c = W.random_cluster(np.random.default_rng(40), 4, 1, 2, 1, U=0.0)
    m = _model(c)
    eps = np.linalg.eigvalsh(m.h)
    L = m.L
    ups = [sum(eps[list(o)]) for o in itertools.combinations(range(L), 2)]
    dns = [sum(eps[list(o)]) for o in itertools.combinations(range(L), 1)]
    levels = np.sort(np.add.outer(ups, dns).ravel())
    E, V = O.low_states(O.sector_hamiltonian(m, 2, 1), 6)
    assert np.allclose(E, levels[:6], atol=1e-11)


def _ring4(t=-1.0, U=3.0):
    T = W.lattice_hopping(4, 1, t=t, periodic=True)
    return W._cluster("4-ring", T, U, 0.0, 2, 0)


def test_mixed_green_of_degenerate_free_states_is_the_resolvent():
    """Two particles of one spin on a 4-site ring (levels 2t cos k: 2t, 0, 0, -2t for t < 0): the
    ground state is doubly degenerate.  For free fermions every eigenstate has G = (z - h)^-1
    (Eq. G0), so the T = 0 mixture over the degenerate pair must give it too."""
    c = _ring4()
    m = _model(c)
    z = np.array([-1.5 + 0.2j, 0.3 + 0.05j, 2.0j, 3.0 + 0.1j])
    G, E, p = O.green_mixed(m, 2, 0, z, k=4)
    assert abs(E[1] - E[0]) < 1e-12 and E[2] - E[0] > 0.5  # doubly degenerate ground state
    assert np.allclose(p, [0.5, 0.5, 0.0, 0.0])
    want = np.linalg.inv(z[:, None, None] * np.eye(4) - m.h[None])
    assert np.max(np.abs(G - want)) <= 1e-12


def test_mixed_green_does_not_depend_on_the_degenerate_basis():
    """Equal weights over a degenerate manifold give a G that is the same for any orthonormal
    basis of it (here a rotated pair), while the Green function of a single state of the pair is
    not unique."""
    c = _ring4(U=2.5)
    c["n_dn"] = 1
    m = _model(c)
    op = O.sector_hamiltonian(m, 2, 1)
    E, V = O.low_states(op, 3)
    assert abs(E[1] - E[0]) < 1e-10, E
    z = 1j * W.matsubara_grid(16, 50.0)
    a = 0.6
    R0 = math.cos(a) * V[0] + math.sin(a) * V[1]
    R1 = -math.sin(a) * V[0] + math.cos(a) * V[1]
    g = lambda s, v: O.green_exact(m, 2, 1, z, state=(E[s], v))[0]
    G_eig = 0.5 * (g(0, V[0]) + g(1, V[1]))
    G_rot = 0.5 * (g(0, R0) + g(1, R1))
    assert np.max(np.abs(G_eig - G_rot)) <= 1e-12
    assert np.max(np.abs(g(0, V[0]) - g(0, R0))) > 1e-6


def test_mixed_green_low_temperature_limit_and_sum_rule():
    """A non-degenerate ground state: at T far below the gap the mixture is the ground-state G;
    at any T the weights sum to one and z G(z) -> 1 (Eq. norm)."""
    c = W.random_cluster(np.random.default_rng(42), 3, 1, 2, 2)
    m = _model(c)
    z = np.concatenate([1j * W.matsubara_grid(8, 50.0), [1e6j]])
    G0, Q, w, E0, gap = O.green_exact(m, 2, 2, z)
    assert gap > 1e-3
    Gm, E, p = O.green_mixed(m, 2, 2, z, k=3, T=gap / 200)
    assert np.max(np.abs(Gm - G0)) <= 1e-12
    Gt, E, p = O.green_mixed(m, 2, 2, z, k=3, T=gap)
    assert abs(p.sum() - 1.0) < 1e-15 and p[1] > 0.1 * p[0]
    assert np.max(np.abs(z[-1] * Gt[-1] - np.eye(3))) <= 1e-5


def test_free_fermion_mixture_at_any_temperature_is_the_resolvent():
    """U = 0: every eigenstate has G = (z - h)^-1 (Eq. G0) when its own energy is the reference,
    so a Boltzmann mixture of the four lowest states at T = 1 must be the resolvent too."""
    c = W.random_cluster(np.random.default_rng(43), 3, 2, 2, 2, U=0.0)
    m = _model(c)
    z = np.array([-1.0 + 0.3j, 0.7 + 0.05j, 2.5j])
    G, E, p = O.green_mixed(m, 2, 2, z, k=4, T=1.0)
    assert np.all(p > 0.01)
    want = np.linalg.inv(z[:, None, None] * np.eye(m.L) - m.h[None])[:, :3, :3]
    assert np.max(np.abs(G - want)) <= 1e-12
