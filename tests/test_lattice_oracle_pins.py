"""Pins of the lattice oracle (oracle/lattice_oracle.py): cluster perturbation theory (Sec. 3) and
the CDMFT bath fit (Sec. 6), each checked against something other than itself: the worked
example printed in Sec. 2.2, closed forms that hold at U = 0 (CPT is exact there, Sec. 3.3), the
Schur complement of the full one-body resolvent, and a real-space lattice built independently
of any Fourier transform."""

import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import lattice_oracle as LO
from paper_2305_18643_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.json")


def _g0(h, z):
    """Non-interacting Green function (z - h)^-1 of Eq. G0 on a grid."""
    L = h.shape[0]
    return np.linalg.inv(np.asarray(z)[:, None, None] * np.eye(L) - h[None])


def test_mixed_hopping_worked_example():
    """Sec. 2.2: a chain with nearest-neighbour hopping (dispersion -2 t cos k) tiled by 2-site
    clusters has t(k~) = -t [[0, 1 + e^{-2ik~}], [1 + e^{2ik~}, 0]].  Here the matrix element of
    the hop is -t."""
    g = json.load(open(GOLDEN))["mixed_hopping_chain_L2"]
    tpar = 1.3
    lat = W.square_superlattice(2, 1, t=-tpar)
    for kt in np.linspace(-np.pi, np.pi, 9):
        want = -tpar * np.array([[0.0, 1 + np.exp(-2j * kt)], [1 + np.exp(2j * kt), 0.0]])
        got = LO.mixed_hopping(lat["t_c"], lat["bonds"], lat["E"], np.array([kt]))
        assert np.allclose(got, want, atol=1e-14), kt
        assert np.allclose(got, got.conj().T)
    assert g["L"] == 2 and g["period"] == 2


@pytest.mark.parametrize("W_,H_,tp", [(2, 1, 0.0), (4, 1, 0.0), (2, 2, 0.0), (2, 2, 0.35)])
def test_cpt_exact_at_u0(W_, H_, tp):
    """CPT is exact at U = 0 (Sec. 3.3): with G_c = (z - t_c)^-1 the periodized CPT Green
    function (Eqs. CPT1, CPT3) is 1 / (z - eps(k)) for the lattice dispersion
    eps(k) = 2 t (cos kx + cos ky) + 2 t' (cos(kx + ky) + cos(kx - ky)), at arbitrary k."""
    t = -1.0
    lat = W.square_superlattice(W_, H_, t=t, tp=tp)
    z = np.array([-1.3 + 0.2j, 0.4 + 0.05j, 2.0 + 1.0j, 0.7j])
    rng = np.random.default_rng(3)
    D = lat["E"].shape[0]
    k = rng.uniform(-np.pi, np.pi, (7, D))
    Gc = _g0(lat["t_c"], z)
    V = LO.inter_cluster(lat["bonds"], lat["t_c"].shape[0], lat["E"], k)
    G = LO.cpt_green(Gc, V)
    Gp = LO.periodize(G, lat["pos"], k)
    if D == 1:
        eps = 2 * t * np.cos(k[:, 0])
    else:
        kx, ky = k[:, 0], k[:, 1]
        eps = 2 * t * (np.cos(kx) + np.cos(ky)) + 2 * tp * (np.cos(kx + ky) + np.cos(kx - ky))
    want = 1.0 / (z[None, :] - eps[:, None])
    assert np.max(np.abs(Gp - want)) <= 1e-12


def test_hybridization_schur_complement():
    """At U = 0 the cluster block of the full resolvent (z - h)^-1 of a cluster with bath
    (Eq. cdmft1) is (z - h_c - Gamma(z))^-1 with Gamma of Eq. hybridization (a Schur complement);
    one bath orbital gives Gamma = theta theta^T / (z - eps) exactly."""
    c = W.random_cluster(np.random.default_rng(5), 3, 4, 2, 2, U=0.0)
    m = O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])
    z = np.array([-2.0 + 0.1j, 0.3 + 0.05j, 1.7j])
    R = _g0(m.h, z)[:, :3, :3]
    Gam = LO.hybridization(c["theta"], c["eps"], z)
    hc = m.h[:3, :3]
    assert np.max(np.abs(np.linalg.inv(R) - (z[:, None, None] * np.eye(3) - hc - Gam))) <= 1e-12
    one = LO.hybridization(c["theta"][:, :1], c["eps"][:1], z)
    want = np.outer(c["theta"][:, 0], c["theta"][:, 0])[None] / (z - c["eps"][0])[:, None, None]
    assert np.max(np.abs(one - want)) <= 1e-15


@pytest.mark.parametrize("W_,H_,ncells", [(4, 1, (6,)), (2, 2, (3, 3)), (3, 1, (5,))])
def test_superlattice_average_real_space(W_, H_, ncells):
    """G_bar (CDMFT step 3) at U = 0 on the reduced-zone grid of a periodic lattice of N clusters
    equals the cluster block of the resolvent of that finite lattice built in real space."""
    lat = W.square_superlattice(W_, H_, t=-1.0, tp=0.25 if H_ > 1 else 0.0)
    L = lat["t_c"].shape[0]
    z = np.array([-1.1 + 0.3j, 0.5 + 0.1j, 2.5j])
    kt = W.reduced_zone(lat["E"], ncells)
    V = LO.inter_cluster(lat["bonds"], L, lat["E"], kt)
    Gbar = LO.superlattice_average(_g0(lat["t_c"], z), V)
    T, cells = LO.real_space_lattice(lat["t_c"], lat["bonds"], ncells)
    Rfull = _g0(T, z)[:, :L, :L]
    assert np.max(np.abs(Gbar - Rfull)) <= 1e-12


def test_self_energy_vanishes_at_u0():
    """Sigma_c = z - h_c - Gamma - G_c^-1 (Sec. 6) of a cluster with bath is zero at U = 0, with
    G_c from the exact-diagonalization oracle (Eq. spectral1 in the N +- 1 sectors)."""
    c = W.random_cluster(np.random.default_rng(6), 2, 3, 2, 2, U=0.0)
    m = O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])
    z = 1j * W.matsubara_grid(16, 50.0)
    Gc, Q, w, E0, gap = O.green_exact(m, 2, 2, z)
    assert gap > 1e-6
    S = LO.self_energy(Gc, z, m.h[:2, :2], LO.hybridization(c["theta"], c["eps"], z))
    assert np.max(np.abs(S)) <= 1e-10


def test_cdmft_distance_zero_at_generating_bath():
    """The distance of Eq. dist_func vanishes when the target calG_0^-1 is the one a bath
    (eps*, theta*) produces, z - h_c - Gamma*(z), and is positive for any other bath."""
    rng = np.random.default_rng(8)
    L, nb = 2, 4
    h_c = np.array([[0.1, -1.0], [-1.0, -0.2]])
    th, ep = rng.uniform(0.2, 0.8, (L, nb)), rng.uniform(-2, 2, nb)
    z = 1j * W.matsubara_grid(64, 50.0)
    Wn = np.ones(len(z))
    G0i = z[:, None, None] * np.eye(L) - h_c - LO.hybridization(th, ep, z)
    A = z[:, None, None] * np.eye(L) - h_c - G0i
    assert LO.cdmft_distance(th, ep, z, Wn, A) <= 1e-26
    assert LO.cdmft_distance(th * 1.01, ep, z, Wn, A) > 1e-8
    assert LO.cdmft_distance(th, ep + 0.01, z, Wn, A) > 1e-8
