"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage or closed form it checks.  Together they are chosen so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle fails one of them.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2305_18643_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _bits(s):
    """Printed occupation string, orbital 0 on the left (Sec. 4.1) -> integer bit string."""
    return sum(1 << i for i, ch in enumerate(s) if ch == "1")


def _model(c):
    return O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])


# ----------------------------------------------------------------------------- basis
@pytest.mark.parametrize("L", range(0, 13))
def test_basis_dimension_and_cns_rank(L):
    """Eq. Hilbert1: d(N) = L!/(N!(L-N)!); label = combinatorial-number-system rank."""
    for N in range(0, L + 1):
        B = O.sector_basis(L, N)
        assert len(B) == math.comb(L, N)
        assert np.all(np.diff(B.astype(np.int64)) > 0)
        assert np.all(O.popcount(B) == N)
        for idx in range(0, len(B), max(1, len(B) // 50)):
            b = int(B[idx])
            pos = [p for p in range(L) if (b >> p) & 1]
            rank = sum(math.comb(p, k + 1) for k, p in enumerate(pos))
            assert rank == idx


def test_paper_dimensions():
    """Table 1 (Sec. 4.5) irrep dimensions add up to C(12,6)^2; Table 3's sector is half of C(14,7)^2."""
    g = GOLDEN["c2v_3x4_irrep_dims"]
    assert len(O.sector_basis(g["L"], g["N"])) ** 2 == sum(g["dims"])
    g = GOLDEN["chain14_symmetric_sector"]
    assert len(O.sector_basis(g["L"], g["N"])) ** 2 == 2 * g["dim"]


# ----------------------------------------------------------------------------- hopping
def test_worked_sign_example():
    """Sec. 4.1: (10010110) -> (10011100), L = 8, element -t_46."""
    g = GOLDEN["sign_example"]
    L, a, b = g["L"], g["a"], g["b"]
    h = np.zeros((L, L))
    h[a, b] = h[b, a] = 0.37
    src, dst = _bits(g["from"]), _bits(g["to"])
    N = bin(src).count("1")
    B = O.sector_basis(L, N)
    K = O.hopping_matrix(h, N).toarray()
    i_src, i_dst = O.basis_index(B, src), O.basis_index(B, dst)
    assert K[i_dst, i_src] == pytest.approx(g["sign"] * 0.37, abs=0)
    assert K[i_src, i_dst] == pytest.approx(g["sign"] * 0.37, abs=0)
    row, col, aa, bb, sign = O.hop_entries(h, N)
    sel = (row == i_dst) & (col == i_src)
    assert sel.sum() == 1 and aa[sel][0] == a and bb[sel][0] == b and sign[sel][0] == g["sign"]


@pytest.mark.parametrize("L,N", [(4, 2), (6, 3), (7, 2), (8, 4), (9, 5)])
def test_nnz_closed_form(L, N):
    """Every ordered pair (a, b), a != b, connects C(L-2, N-1) states."""
    rng = np.random.default_rng(L * 10 + N)
    h = rng.uniform(0.1, 1.0, (L, L))
    row, col, a, b, sign = O.hop_entries(h, N)
    assert len(row) == L * (L - 1) * math.comb(L - 2, N - 1)


@pytest.mark.parametrize("seed,ns,nb,nu,nd", [(1, 2, 1, 1, 2), (2, 3, 1, 2, 2), (3, 2, 2, 2, 1),
                                               (4, 3, 2, 3, 2), (5, 4, 0, 2, 3), (6, 5, 0, 2, 2)])
def test_factorized_matches_jordan_wigner(seed, ns, nb, nu, nd):
    """Eq. factorized with the (-1)^{M_ab} rule equals the generic Jordan-Wigner Hamiltonian
    built in the global ordering of Eq. basis, element by element (non-symmetric h too,
    which exposes a transposed operand)."""
    rng = np.random.default_rng(seed)
    c = W.random_cluster(rng, ns, nb, nu, nd, dense_t=True)
    m = _model(c)
    for h in (m.h, m.h + np.triu(rng.uniform(-0.3, 0.3, m.h.shape), 1)):
        m.h = h
        Hjw = O.jw_hamiltonian_dense(m, nu, nd)
        Hf = O.sector_hamiltonian(m, nu, nd).sparse().toarray()
        assert np.max(np.abs(Hjw - Hf)) < 1e-13


def test_sampled_matvec_matches_full():
    c = W.random_cluster(np.random.default_rng(9), 4, 2, 3, 2)
    op = O.sector_hamiltonian(_model(c), 3, 2)
    psi = np.random.default_rng(1).standard_normal(op.shape2)
    y = O.apply_h(op, psi)
    us = np.arange(op.shape2[0]).repeat(3)[: 40]
    ds = (np.arange(len(us)) * 7) % op.shape2[1]
    assert np.allclose(O.apply_h_sampled(op, psi, us, ds), y[us, ds], atol=1e-13)
    rows = np.array([0, 2, op.shape2[0] - 1])
    assert np.allclose(O.apply_h_rows(_model(c), 3, 2, psi, rows), y[rows], atol=1e-13)
    H = op.sparse()
    assert abs(H - H.T).max() < 1e-14


# ----------------------------------------------------------------------------- ground state
@pytest.mark.parametrize("t,U,mu", [(-1.0, 4.0, 0.0), (-1.0, 8.0, 4.0), (0.7, 2.5, 1.3), (-1.3, 0.0, 0.0)])
def test_two_site_closed_form(t, U, mu):
    """Half-filled dimer: E0 = (U - sqrt(U^2 + 16 t^2)) / 2 - 2 mu."""
    c = W.hubbard_dimer(t, U, mu)
    m = _model(c)
    E0, _, _ = O.ground_state(O.sector_hamiltonian(m, 1, 1))
    ref = 0.5 * (U - math.sqrt(U * U + 16 * t * t)) - 2 * mu
    assert E0 == pytest.approx(ref, abs=1e-13)
    Ejw = np.linalg.eigvalsh(O.jw_hamiltonian_dense(m, 1, 1))[0]
    assert Ejw == pytest.approx(ref, abs=1e-13)


@pytest.mark.parametrize("seed,ns,nb,nu,nd", [(11, 4, 2, 3, 2), (12, 6, 0, 3, 3), (13, 3, 3, 2, 4), (14, 4, 4, 4, 4)])
def test_free_fermion_ground_energy(seed, ns, nb, nu, nd):
    """U = 0: E0 = sum of the lowest N_up plus the lowest N_dn eigenvalues of h (Sec. 3.1)."""
    c = W.random_cluster(np.random.default_rng(seed), ns, nb, nu, nd, U=0.0)
    m = _model(c)
    eps = np.linalg.eigvalsh(m.h)
    E0, _, _ = O.ground_state(O.sector_hamiltonian(m, nu, nd))
    assert E0 == pytest.approx(eps[:nu].sum() + eps[:nd].sum(), abs=1e-11)


@pytest.mark.parametrize("mu,eps,theta", [(1.0, -0.5, 0.7), (-0.3, 1.2, 0.4), (2.0, 2.0, 1.0)])
def test_site_bath_pair_closed_form(mu, eps, theta):
    """One site (on-site energy -mu) hybridized with one bath orbital (energy eps, coupling
    theta, Eq. cdmft1), U = 0: the one-body levels are (e_s + eps)/2 -+ sqrt(((e_s - eps)/2)^2
    + theta^2) with e_s = -mu, so E0 = 2 l_min with one electron of each spin and l_min with
    one up electron alone."""
    es = -mu
    lmin = 0.5 * (es + eps) - math.sqrt((0.5 * (es - eps)) ** 2 + theta * theta)
    for nu, nd, ref in ((1, 1, 2 * lmin), (1, 0, lmin)):
        c = W._cluster("site+bath", np.zeros((1, 1)), 0.0, mu, nu, nd, eps=[eps], theta=[[theta]])
        E0, _, _ = O.ground_state(O.sector_hamiltonian(_model(c), nu, nd))
        assert E0 == pytest.approx(ref, abs=1e-13)


@pytest.mark.parametrize("L,nu,nd,U,mu", [(6, 3, 3, 4.0, 2.0), (6, 4, 4, 3.0, 1.0), (7, 5, 3, 5.0, 0.5), (5, 1, 2, 2.0, -1.0)])
def test_atomic_limit(L, nu, nd, U, mu):
    """t = 0: E0 = U max(0, N_up + N_dn - L) - mu (N_up + N_dn) for U > 0 (fewest double occupations)."""
    c = W._cluster("atomic", np.zeros((L, L)), U, mu, nu, nd)
    E0, _, _ = O.ground_state(O.sector_hamiltonian(_model(c), nu, nd))
    assert E0 == pytest.approx(U * max(0, nu + nd - L) - mu * (nu + nd), abs=1e-13)


def test_dense_and_sparse_eigensolvers_agree():
    c = W.random_cluster(np.random.default_rng(21), 4, 3, 3, 4)
    op = O.sector_hamiltonian(_model(c), 3, 4)
    Ed, Od, _ = O.ground_state(op)
    Es, Os, _ = O.ground_state(op, dense_limit=0)
    assert Es == pytest.approx(Ed, abs=1e-11)
    assert abs(abs(np.vdot(Od, Os)) - 1) < 1e-9


# ----------------------------------------------------------------------------- Green function
Z = np.concatenate([W.real_grid(41, -6, 6) + 0.3j, 1j * W.matsubara_grid(20, 10.0)])


@pytest.mark.parametrize("seed,ns,nb,nu,nd", [(31, 4, 2, 2, 3), (32, 3, 2, 2, 2), (33, 5, 0, 2, 2)])
def test_green_free_fermions(seed, ns, nb, nu, nd):
    """U = 0 with a non-degenerate Fermi level: G(z) = [(z - h)^{-1}]_{sites} (Eq. G0), for
    the exact Lehmann sum, the continued fractions and the band Lanczos representation."""
    c = W.random_cluster(np.random.default_rng(seed), ns, nb, nu, nd, U=0.0)
    m = _model(c)
    eps = np.linalg.eigvalsh(m.h)
    assert eps[nu] - eps[nu - 1] > 1e-3
    ref = np.stack([np.linalg.inv(z * np.eye(m.L) - m.h)[:ns, :ns] for z in Z])
    Ge = O.green_exact(m, nu, nd, Z)[0]
    Gc = O.green_cf(m, nu, nd, Z)[0]
    Gb = O.green_band(m, nu, nd, Z)[0]
    for G in (Ge, Gc, Gb):
        assert np.max(np.abs(G - ref)) < 1e-10


@pytest.mark.parametrize("nu,nd,U,mu,pole", [(0, 1, 5.0, 1.5, "U-mu"), (1, 1, 5.0, 1.5, "U-mu"), (1, 0, 5.0, 1.5, "-mu")])
def test_one_site_atomic_green(nu, nd, U, mu, pole):
    """One site: G_up(z) = 1/(z - (U - mu)) when adding to / removing from a doubly
    occupiable site, 1/(z + mu) when removing the only electron (electron pole E_r - E0,
    hole pole E0 - E_r, Eq. spectral1)."""
    c = W._cluster("atom", np.zeros((1, 1)), U, mu, nu, nd)
    G = O.green_exact(_model(c), nu, nd, Z)[0][:, 0, 0]
    w = U - mu if pole == "U-mu" else -mu
    assert np.max(np.abs(G - 1.0 / (Z - w))) < 1e-13
    Gc = O.green_cf(_model(c), nu, nd, Z)[0][:, 0, 0]
    assert np.max(np.abs(Gc - 1.0 / (Z - w))) < 1e-13


@pytest.mark.parametrize("seed,ns,nb,nu,nd", [(41, 3, 3, 3, 2), (42, 4, 2, 3, 3), (43, 4, 0, 2, 2)])
def test_green_sum_rules_and_methods(seed, ns, nb, nu, nd):
    """Interacting clusters: Q Q^T = 1 (Eq. norm); first moment sum_r Q_ir^2 w_r = h_ii +
    U_i <n_{i dn}> (from {[c_i, H], c+_i}); G_ij = G_ji; z G(z) -> 1; continued fractions
    and band Lanczos agree with the exact Lehmann sum."""
    c = W.random_cluster(np.random.default_rng(seed), ns, nb, nu, nd)
    m = _model(c)
    G, Q, w, E0, gap = O.green_exact(m, nu, nd, Z)
    assert gap > 1e-6
    assert np.max(np.abs(Q @ Q.T - np.eye(ns))) < 1e-12
    _, Om, _ = O.ground_state(O.sector_hamiltonian(m, nu, nd))
    n_dn = O.density(m, nu, nd, Om, 1)
    m1 = (Q * Q) @ w
    assert np.max(np.abs(m1 - (np.diag(m.h)[:ns] + m.U[:ns] * n_dn[:ns]))) < 1e-11
    assert np.max(np.abs(G - G.transpose(0, 2, 1))) < 1e-13
    zbig = np.array([1e7j, -3e7 + 1e6j])
    Gbig = O.lehmann_green(Q, w, zbig)
    assert np.max(np.abs(zbig[:, None, None] * Gbig - np.eye(ns))) < 1e-5
    Gc, coeffs = O.green_cf(m, nu, nd, Z)
    assert np.max(np.abs(Gc - G)) < 1e-10
    for x in range(ns):
        assert coeffs[("e", x, x)][1][0] + coeffs[("h", x, x)][1][0] == pytest.approx(1.0, abs=1e-13)
    Gb = O.green_band(m, nu, nd, Z)[0]
    assert np.max(np.abs(Gb - G)) < 1e-10


def test_green_spin_symmetry():
    """N_up = N_dn and a spin-symmetric H: G_up = G_dn (checks the down-spin operator sign)."""
    c = W.random_cluster(np.random.default_rng(51), 3, 2, 2, 2)
    m = _model(c)
    Gu = O.green_exact(m, 2, 2, Z, spin=0)[0]
    Gd = O.green_exact(m, 2, 2, Z, spin=1)[0]
    assert np.max(np.abs(Gu - Gd)) < 1e-12


def test_cf_without_reorthogonalization_converges():
    """The paper's three-vector recursion (no reorthogonalization) reproduces G at eta = 0.05
    once it runs past the sector dimension: the ghost copies of Sec. 4.2 carry no weight in
    the continued fraction.  At exactly the dimension (300) it is still off by ~1e-6."""
    c = W.random_cluster(np.random.default_rng(61), 4, 2, 3, 3)
    m = _model(c)
    z = W.real_grid(101) + 0.05j
    Ge = O.green_exact(m, 3, 3, z)[0]
    Gc = O.green_cf(m, 3, 3, z, reorth=False, max_steps=600, btol=0.0)[0]
    assert np.max(np.abs(Gc - Ge)) < 1e-11


def test_ladder14_golden_properties():
    """The stored 2x7 reference (tests/golden/make_ladder14.py, oracle only): G_ij = G_ji for a
    real H (Sec. 4.3), Im G_ii(i omega) < 0 for omega > 0 (positive spectral weight, Eq. spectral1),
    G_ii(i omega) purely damped toward -i/omega (its magnitude below 1/omega, Eq. norm), and an E0
    below the ladder's atomic-limit energy with every hop removed (a variational bound)."""
    import os
    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ladder14_band.npz"))
    G, om = g["G"], g["omega"]
    assert np.max(np.abs(G - G.transpose(0, 2, 1))) <= 1e-12
    d = np.einsum("kii->ki", G)
    assert np.all(d.imag < 0)
    assert np.all(np.abs(d) <= 1.0 / om[:, None] + 1e-12)
    c = W.served_request(np.random.default_rng(int(g["seed"])), sizes=(14,))
    assert float(g["E0"]) < -c["mu"] * 14  # below the atomic state with one electron per site (U n n = 0)
