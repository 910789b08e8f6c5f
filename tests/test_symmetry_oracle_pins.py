"""Pins of the cluster-symmetry oracle (Sec. 4.5) against what the paper and the mathematics fix:

* Table 1: the four C2v subspace dimensions of the half-filled 3x4 cluster and the number of
  nearest-neighbour hopping matrix elements of every value in each of them (24 integers);
* the spectrum of an unsymmetrized sector is the union of the spectra of its irreps (clusters
  with interaction, bath orbitals, asymmetric fillings, a periodic ring with a half translation);
* the dimension of every irrep equals the character formula (1/|G|) sum_g chi_g^* Tr(g);
* groups with complex characters (C4 rotations, translations of rings, Z4 x Z2 of a periodic
  ladder): Hermitian irrep matrices whose spectra make up the sector's;
* an irrep eigenvector written back in the unsymmetrized sector is an eigenvector of the full H
  with the same energy, on which every group element acts as its character;
* planted mistakes (no fermionic phase, no character, no stabilizer factor) fail these pins.
"""

import json
import os

import numpy as np
import pytest

import oracle.symmetry_oracle as S
from oracle.ed_oracle import Model, apply_h, jw_hamiltonian_dense, sector_hamiltonian

HERE = os.path.dirname(os.path.abspath(__file__))


def rect(W, H, t=-1.0):
    L = W * H
    h = np.zeros((L, L))
    for y in range(H):
        for x in range(W):
            s = x + W * y
            if x + 1 < W:
                h[s, s + 1] = h[s + 1, s] = t
            if y + 1 < H:
                h[s, s + W] = h[s + W, s] = t
    mx = [(W - 1 - s % W) + W * (s // W) for s in range(L)]
    my = [s % W + W * (H - 1 - s // W) for s in range(L)]
    return h, mx, my


def _cases():
    """(name, model, n_up, n_dn, generators) for the spectrum pins."""
    out = []
    h, mx, my = rect(3, 2)
    out.append(("2x3 C2v U=4", Model(h, 4.0, 2.0), 3, 3, [mx, my]))
    out.append(("2x3 mirror, N_up != N_dn", Model(h, 3.0, 1.0), 2, 3, [mx]))
    # 6-site chain with a second-neighbour hop, inversion
    L = 6
    t = np.zeros((L, L))
    for i in range(L - 1):
        t[i, i + 1] = t[i + 1, i] = -1.0
    for i in range(L - 2):
        t[i, i + 2] = t[i + 2, i] = 0.3
    inv = [L - 1 - i for i in range(L)]
    out.append(("chain6 inversion", Model(t, 5.0, 2.5), 3, 2, [inv]))
    # periodic 4-ring: half translation and inversion (commuting involutions)
    t = np.zeros((4, 4))
    for i in range(4):
        t[i, (i + 1) % 4] = t[(i + 1) % 4, i] = -1.0
    T2 = [(i + 2) % 4 for i in range(4)]
    I4 = [(-i) % 4 for i in range(4)]
    out.append(("ring4 T2 x I", Model(t, 6.0, 3.0), 2, 2, [T2, I4]))
    out.append(("ring4 T2, odd filling", Model(t, 6.0, 3.0), 1, 2, [T2]))
    # 2x2 plaquette with one bath orbital per site; the mirrors permute sites and baths alike
    h, mx, my = rect(2, 2)
    h[0, 3] = h[3, 0] = h[1, 2] = h[2, 1] = 0.3
    eps = np.array([-1.0, -1.0, -1.0, -1.0])
    theta = 0.5 * np.eye(4)
    mxb = mx + [4 + mx[a] for a in range(4)]
    myb = my + [4 + my[a] for a in range(4)]
    out.append(("plaquette + bath C2v", Model(h, 8.0, 4.0, eps, theta), 3, 3, [mxb, myb]))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_irrep_spectra_make_up_the_sector_spectrum(case):
    name, m, nu, nd, gens = case
    full = np.linalg.eigvalsh(jw_hamiltonian_dense(m, nu, nd))
    parts = S.irrep_spectra(m, nu, nd, gens)
    union = np.sort(np.concatenate(list(parts.values())))
    assert union.shape == full.shape
    assert np.max(np.abs(union - full)) < 1e-10 * max(1.0, np.max(np.abs(full)))


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_irrep_dimensions_follow_the_character_formula(case):
    name, m, nu, nd, gens = case
    tot = 0
    for ir in S.all_irreps(len(gens)):
        bu, bd, st = S.symmetric_basis(m.L, nu, nd, gens, ir)
        assert len(bu) == S.irrep_dimension_formula(m.L, nu, nd, gens, ir)
        tot += len(bu)
        key = (bu.astype(np.uint64) << np.uint64(m.L)) | bd.astype(np.uint64)
        assert np.all(np.diff(key.astype(np.float64)) > 0)  # ascending, distinct
        assert set(np.unique(st).tolist()) <= {1, 2, 4, 8}
    from math import comb

    assert tot >= comb(m.L, nu) * comb(m.L, nd) // (1 << len(gens))


def test_table1_c2v_3x4_dimensions_and_matrix_element_counts():
    """Table 1: every dimension and every count of the nearest-neighbour hopping operator."""
    ref = json.load(open(os.path.join(HERE, "golden", "table1_c2v_3x4.json")))
    h, mx, my = rect(4, 3)
    m = Model(h, 0.0, 0.0)
    names = {"-2": -2.0, "-sqrt2": -np.sqrt(2.0), "-1": -1.0, "1": 1.0, "sqrt2": np.sqrt(2.0), "2": 2.0}
    total = 0
    for label, signs in ref["irreps_by_generator_signs"].items():
        H, (bu, bd, st) = S.symmetric_hamiltonian(m, 6, 6, [mx, my], tuple(signs))
        assert H.shape[0] == ref["dim"][label]
        total += H.shape[0]
        assert abs(H - H.T).max() == 0.0
        for name, v in names.items():
            assert int(np.sum(np.abs(H.data - v) < 1e-12)) == ref["counts"][label][name], (label, name)
        assert H.nnz == sum(ref["counts"][label].values())  # no other value occurs
    assert total == 924 * 924


def _complex_cases():
    """(name, model, n_up, n_dn, generators, orders): groups with complex characters."""
    out = []
    # periodic 4-ring: translation by one site (order 4: the momenta 0, pi/2, pi, 3pi/2)
    t = np.zeros((4, 4))
    for i in range(4):
        t[i, (i + 1) % 4] = t[(i + 1) % 4, i] = -1.0
    out.append(("ring4 C4 translation", Model(t, 5.0, 2.5), 2, 2, [[(i + 1) % 4 for i in range(4)]], (4,)))
    out.append(("ring4 C4, odd filling", Model(t, 5.0, 2.5), 1, 2, [[(i + 1) % 4 for i in range(4)]], (4,)))
    # periodic 6-ring with a second-neighbour hop: translation of order 6
    t = np.zeros((6, 6))
    for i in range(6):
        t[i, (i + 1) % 6] = t[(i + 1) % 6, i] = -1.0
        t[i, (i + 2) % 6] = t[(i + 2) % 6, i] = 0.3
    out.append(("ring6 translation", Model(t, 4.0, 2.0), 3, 2, [[(i + 1) % 6 for i in range(6)]], (6,)))
    # 2x2 plaquette with diagonals and one bath orbital per site: the four-fold rotation
    h, _, _ = rect(2, 2)
    h[0, 3] = h[3, 0] = h[1, 2] = h[2, 1] = 0.3
    rot = [1, 3, 0, 2]  # (x, y) -> (1 - y, x) on s = x + 2 y
    out.append(("plaquette + bath C4", Model(h, 8.0, 4.0, np.full(4, -1.0), 0.5 * np.eye(4)), 3, 3,
                [rot + [4 + v for v in rot]], (4,)))
    # 2-leg ladder periodic along the legs (4 rungs): translation (order 4) x leg exchange
    t = np.zeros((8, 8))
    for x in range(4):
        t[x, (x + 1) % 4] = t[(x + 1) % 4, x] = -1.0
        t[4 + x, 4 + (x + 1) % 4] = t[4 + (x + 1) % 4, 4 + x] = -1.0
        t[x, 4 + x] = t[4 + x, x] = -0.5
    tr = [(s + 1) % 4 + 4 * (s // 4) for s in range(8)]
    leg = [(s + 4) % 8 for s in range(8)]
    out.append(("ladder 2x4 periodic Z4 x Z2", Model(t, 3.0, 1.5), 3, 3, [tr, leg], (4, 2)))
    return out


@pytest.mark.parametrize("case", _complex_cases(), ids=lambda c: c[0])
def test_complex_character_spectra_and_dimensions(case):
    """Groups with complex characters: every irrep's H is Hermitian, its dimension follows the
    character formula, and the irrep spectra make up the unsymmetrized spectrum."""
    name, m, nu, nd, gens, orders = case
    full = np.linalg.eigvalsh(jw_hamiltonian_dense(m, nu, nd))
    parts = []
    for ir in S.all_irreps(len(gens), orders):
        H, (bu, bd, st) = S.symmetric_hamiltonian(m, nu, nd, gens, ir, orders)
        assert H.shape[0] == S.irrep_dimension_formula(m.L, nu, nd, gens, ir, orders)
        if H.shape[0]:
            A = H.toarray()
            assert np.max(np.abs(A - A.conj().T)) < 1e-13
            parts.append(np.linalg.eigvalsh(A))
    union = np.sort(np.concatenate(parts))
    assert union.shape == full.shape
    assert np.max(np.abs(union - full)) < 1e-10 * max(1.0, np.max(np.abs(full)))


@pytest.mark.parametrize("case", _complex_cases() + [c + (None,) for c in _cases()[:3]], ids=lambda c: c[0])
def test_irrep_eigenvectors_embed_as_eigenvectors_with_the_character(case):
    """The lowest eigenvector of every irrep, written back in the unsymmetrized sector from the
    definition of the symmetrized states, is a normalized eigenvector of the full H with the same
    energy, and every generator g acts on it as chi(g): this fixes the phases of the basis and
    the labelling of the irreps, which the spectra alone do not (irreps m and -m of a real H have
    the same spectrum)."""
    name, m, nu, nd, gens, orders = case
    op = sector_hamiltonian(m, nu, nd)
    for ir in S.all_irreps(len(gens), orders):
        H, basis = S.symmetric_hamiltonian(m, nu, nd, gens, ir, orders)
        if H.shape[0] == 0:
            continue
        w, V = np.linalg.eigh(H.toarray())
        psi = S.embed(V[:, 0], basis, m.L, nu, nd, gens, ir, orders)
        assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
        Hpsi = apply_h(op, psi.real) + 1j * apply_h(op, psi.imag)
        assert np.linalg.norm(Hpsi - w[0] * psi) < 1e-10 * max(1.0, abs(w[0]))
        # the labelling convention: generator k acts as exp(2 pi i m_k / n_k) (signs s_k for
        # involutions named by signs)
        for k, gk in enumerate(gens):
            chi = ir[k] if orders is None else np.exp(2j * np.pi * ir[k] / orders[k])
            gpsi = S.apply_group_element(psi, np.asarray(gk), m.L, nu, nd)
            assert np.linalg.norm(gpsi - chi * psi) < 1e-12, (ir, k)


def test_complex_characters_reduce_to_signs_for_involutions():
    """Order-2 generators named by exponents (0, 1) give the same matrices as the sign names."""
    h, mx, my = rect(3, 2)
    m = Model(h, 4.0, 2.0)
    for signs, exps in (((1, 1), (0, 0)), ((1, -1), (0, 1)), ((-1, -1), (1, 1))):
        A, _ = S.symmetric_hamiltonian(m, 3, 3, [mx, my], signs)
        B, _ = S.symmetric_hamiltonian(m, 3, 3, [mx, my], exps, orders=(2, 2))
        assert A.shape == B.shape
        assert np.max(np.abs(A.toarray() - B.toarray())) < 1e-14


# ---- planted mistakes: each must break a pin (checked on the cheap spectrum cases)

def _spectra_ok(case):
    name, m, nu, nd, gens = case
    full = np.linalg.eigvalsh(jw_hamiltonian_dense(m, nu, nd))
    parts = S.irrep_spectra(m, nu, nd, gens)
    union = np.sort(np.concatenate(list(parts.values())))
    return union.shape == full.shape and np.max(np.abs(union - full)) < 1e-10 * max(1.0, np.max(np.abs(full)))


@pytest.mark.parametrize("mutation", ["no_phase", "no_character", "no_stabilizer_factor"])
def test_planted_mistakes_fail_the_spectrum_pins(monkeypatch, mutation):
    cases = [_cases()[0], _cases()[3], _cases()[5]]
    assert all(_spectra_ok(c) for c in cases)
    if mutation == "no_phase":
        monkeypatch.setattr(S, "perm_sign", lambda p, b: np.ones(np.asarray(b).shape, dtype=np.int64))
    elif mutation == "no_character":
        monkeypatch.setattr(S, "character", lambda *a, **k: 1)
    else:
        real = S.symmetric_basis

        def flat(*a, **k):
            bu, bd, st = real(*a, **k)
            return bu, bd, np.ones_like(st)

        monkeypatch.setattr(S, "symmetric_basis", flat)
    assert not all(_spectra_ok(c) for c in cases)
