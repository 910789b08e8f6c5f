"""Symmetrized sectors (Sec. 4.5) on the GPU against the symmetry oracle: the representatives and
their stabilizers bit for bit, the stored matrix entry by entry, H.psi, and the ground energy of
every irrep; Table 1's counts straight from the device matrix; invalid groups are refused; the
Green function with symmetrized operators (Sec. 4.6) against the exact Lehmann sum; the same for
Abelian groups with complex characters (rotations of order 4, ring translations)."""

import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle.symmetry_oracle as S
import oracle_memo as OM
from oracle.ed_oracle import Model
from paper_2305_18643_gb300 import build, ed

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def libed():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return ed.lib()


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


def _cluster(t, U, mu, nu, nd, eps=None, theta=None, seed=11):
    t = np.asarray(t, dtype=np.float64)
    ns = t.shape[0]
    c = {"t": t, "U": np.full(ns, float(U)), "mu": float(mu), "n_up": nu, "n_dn": nd}
    if eps is not None:
        c["eps"] = np.asarray(eps, dtype=np.float64)
        c["theta"] = np.asarray(theta, dtype=np.float64)
    return ed.ed_cluster_create(c, precision=ed.ED_FP64, seed=seed, tol=1e-13, max_iter=600), \
        Model(t, U, mu, eps, theta)


def _cases():
    out = []
    h, mx, my = rect(3, 2)
    out.append(("2x3 C2v U=4", (h, 4.0, 2.0, 3, 3), [mx, my]))
    out.append(("2x3 mirror N_up != N_dn", (h, 3.0, 1.0, 2, 3), [mx]))
    L = 6
    t = np.zeros((L, L))
    for i in range(L - 1):
        t[i, i + 1] = t[i + 1, i] = -1.0
    for i in range(L - 2):
        t[i, i + 2] = t[i + 2, i] = 0.3
    out.append(("chain6 inversion", (t, 5.0, 2.5, 3, 2), [[L - 1 - i for i in range(L)]]))
    t = np.zeros((4, 4))
    for i in range(4):
        t[i, (i + 1) % 4] = t[(i + 1) % 4, i] = -1.0
    out.append(("ring4 T2 x I", (t, 6.0, 3.0, 2, 2), [[(i + 2) % 4 for i in range(4)], [(-i) % 4 for i in range(4)]]))
    h, mx, my = rect(4, 2)
    h[0, 5] = h[5, 0] = h[1, 4] = h[4, 1] = h[1, 6] = h[6, 1] = h[2, 5] = h[5, 2] = 0.3
    h[2, 7] = h[7, 2] = h[3, 6] = h[6, 3] = 0.3
    out.append(("2x4 t' C2v", (h, 8.0, 4.0, 4, 4), [mx, my]))
    return out


def _bath_case():
    h, mx, my = rect(2, 2)
    h[0, 3] = h[3, 0] = h[1, 2] = h[2, 1] = 0.3
    eps = np.full(4, -1.0)
    theta = 0.5 * np.eye(4)
    return (h, 8.0, 4.0, 3, 3, eps, theta), [mx + [4 + v for v in mx], my + [4 + v for v in my]]


def _device_csr(s):
    d, z = ed.ed_sym_info(s)
    rp, col, val = ed.ed_sym_matrix(s)
    return sp.csr_matrix((val, col, rp), shape=(d, d))


def _check_irrep(hc, m, L, nu, nd, gens, ir):
    s = ed.ed_sym_create(hc, np.array(gens), ir)
    try:
        bu, bd, st = S.symmetric_basis(L, nu, nd, gens, ir)
        keys, stab = ed.ed_sym_basis(s)
        okey = (bu.astype(np.uint64) << np.uint64(L)) | bd.astype(np.uint64)
        assert np.array_equal(keys, okey)
        assert np.array_equal(stab.astype(np.int64), st)
        if len(keys) == 0:
            return None
        Ho, _ = S.symmetric_hamiltonian(m, nu, nd, gens, ir)
        Hg = _device_csr(s)
        assert Hg.nnz == Ho.nnz
        assert np.array_equal(Hg.indptr, Ho.indptr) and np.array_equal(Hg.indices, Ho.indices)
        assert np.max(np.abs(Hg.data - Ho.data)) <= 1e-14 * max(1.0, np.max(np.abs(Ho.data)))
        # H.psi through the C ABI on device vectors
        x = np.random.default_rng(len(keys)).standard_normal(len(keys))
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        ed.ed_sym_hpsi(s, xd.data_ptr(), yd.data_ptr())
        y = yd.cpu().numpy()
        assert np.max(np.abs(y - Ho @ x)) <= 1e-13 * max(1.0, np.max(np.abs(Ho @ x)))
        E, res, it, st_ = ed.ed_sym_ground_state(s)
        Eo = OM.irrep_ground_energy(Ho, m, nu, nd, gens, ir)
        assert abs(E - Eo) <= 1e-10 * max(1.0, abs(Eo)), (E, Eo)
        assert res <= 1e-12 * max(1.0, abs(E))
        w = ed.ed_sym_ground_vector(s)
        assert abs(np.linalg.norm(w) - 1.0) < 1e-12
        assert np.linalg.norm(Ho @ w - E * w) <= 1e-11 * max(1.0, abs(E))
        return E
    finally:
        ed.ed_sym_destroy(s)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_symmetrized_sector_matches_oracle(case):
    name, (t, U, mu, nu, nd), gens = case
    hc, m = _cluster(t, U, mu, nu, nd)
    try:
        Es = [e for ir in S.all_irreps(len(gens)) if (e := _check_irrep(hc, m, m.L, nu, nd, gens, ir)) is not None]
        # the lowest irrep energy is the sector's ground energy
        E0, _, _ = OM.ground_state(m, nu, nd)
        assert abs(min(Es) - E0) <= 1e-10 * max(1.0, abs(E0))
    finally:
        ed.ed_cluster_destroy(hc)


def test_symmetrized_sector_with_bath_orbitals():
    (t, U, mu, nu, nd, eps, theta), gens = _bath_case()
    hc, m = _cluster(t, U, mu, nu, nd, eps, theta)
    try:
        for ir in S.all_irreps(2):
            _check_irrep(hc, m, m.L, nu, nd, gens, ir)
    finally:
        ed.ed_cluster_destroy(hc)


def test_table1_counts_from_the_device_matrix():
    """Table 1 (Sec. 4.5): dimensions and value counts of the nearest-neighbour hopping operator on
    the half-filled 3x4 cluster, read from the matrices the GPU builds."""
    ref = json.load(open(os.path.join(HERE, "golden", "table1_c2v_3x4.json")))
    h, mx, my = rect(4, 3)
    hc, m = _cluster(h, 0.0, 0.0, 6, 6)
    vals = {"-2": -2.0, "-sqrt2": -np.sqrt(2.0), "-1": -1.0, "1": 1.0, "sqrt2": np.sqrt(2.0), "2": 2.0}
    try:
        for label, signs in ref["irreps_by_generator_signs"].items():
            s = ed.ed_sym_create(hc, np.array([mx, my]), signs)
            try:
                d, z = ed.ed_sym_info(s)
                assert d == ref["dim"][label]
                _, _, v = ed.ed_sym_matrix(s)
                for name, x in vals.items():
                    assert int(np.sum(np.abs(v - x) < 1e-12)) == ref["counts"][label][name], (label, name)
                assert z == sum(ref["counts"][label].values())
            finally:
                ed.ed_sym_destroy(s)
    finally:
        ed.ed_cluster_destroy(hc)


def test_3x4_ground_energy_in_a1_matches_the_full_sector():
    """Interacting half-filled 3x4 cluster (U = 4): the A1 ground energy from the 213,840-state
    symmetrized sector against ARPACK on the unsymmetrized 853,776-state sector (oracle), and the
    device matrix against the oracle's."""
    h, mx, my = rect(4, 3)
    hc, m = _cluster(h, 4.0, 2.0, 6, 6)
    try:
        s = ed.ed_sym_create(hc, np.array([mx, my]), [1, 1])
        try:
            Ho, _ = S.symmetric_hamiltonian(m, 6, 6, [mx, my], (1, 1))
            Hg = _device_csr(s)
            assert np.array_equal(Hg.indices, Ho.indices)
            assert np.max(np.abs(Hg.data - Ho.data)) <= 1e-13
            E, res, it, st = ed.ed_sym_ground_state(s)
            E0, _, _ = OM.ground_state(m, 6, 6)
            Ea1 = OM.irrep_ground_energy(Ho, m, 6, 6, [mx, my], (1, 1))
            assert abs(E - Ea1) <= 1e-10 * abs(Ea1)
            assert E >= E0 - 1e-10 * abs(E0)
            assert res <= 1e-12 * max(1.0, abs(E))
        finally:
            ed.ed_sym_destroy(s)
    finally:
        ed.ed_cluster_destroy(hc)


def test_invalid_groups_are_refused():
    h, mx, my = rect(3, 2)
    hc, m = _cluster(h, 4.0, 2.0, 3, 3)
    L = 6
    try:
        bad = [
            ([[1, 2, 0, 4, 5, 3]], [1]),                 # not an involution
            ([[1, 0, 2, 3, 4, 5]], [1]),                 # does not leave h invariant
            ([mx, mx], [1, 1]),                          # dependent generators
            ([mx], [2]),                                 # not a sign
            ([[0, 0, 2, 3, 4, 5]], [1]),                 # not a permutation
        ]
        for perms, signs in bad:
            with pytest.raises(ed.EDError) as e:
                ed.ed_sym_create(hc, np.array(perms), signs)
            assert e.value.status == ed.ED_ERR_INVALID
    finally:
        ed.ed_cluster_destroy(hc)


def _ground_irrep(hc, gens):
    """The irrep holding the sector's ground state: (signs, handle with its ground state, E)."""
    best = None
    for ir in S.all_irreps(len(gens)):
        s = ed.ed_sym_create(hc, np.array(gens), ir)
        d, _ = ed.ed_sym_info(s)
        if d == 0:
            ed.ed_sym_destroy(s)
            continue
        E = ed.ed_sym_ground_state(s)[0]
        if best is None or E < best[2]:
            if best is not None:
                ed.ed_sym_destroy(best[1])
            best = (ir, s, E)
        else:
            ed.ed_sym_destroy(s)
    return best


def _gf_cases():
    out = [c for c in _cases()]
    (t, U, mu, nu, nd, eps, theta), gens = _bath_case()
    out.append(("plaquette + bath C2v", (t, U, mu, nu, nd, eps, theta), gens))
    return out


@pytest.mark.parametrize("case", _gf_cases(), ids=lambda c: c[0])
def test_symmetrized_green_function_matches_oracle(case):
    """Sec. 4.6: G from the irrep ground state with symmetrized site operators, continued
    fractions in the N +- 1 irrep sectors and the M^-1 recombination, against the exact Lehmann
    sum of the unsymmetrized sectors (real axis, eta = 0.1, and Matsubara axis, beta = 50), for
    both spins when N_up != N_dn.  Clusters whose ground state is degenerate are skipped (G is
    then not unique)."""
    name, params, gens = case
    t, U, mu, nu, nd = params[:5]
    eps, theta = (params[5], params[6]) if len(params) > 5 else (None, None)
    hc, m = _cluster(t, U, mu, nu, nd, eps, theta)
    try:
        ir, s, E = _ground_irrep(hc, gens)
        try:
            om_r = np.linspace(-8.0, 8.0, 64)
            om_m = (2 * np.arange(32) + 1) * np.pi / 50.0
            for spin in ((0, 1) if nu != nd else (0,)):
                Gr, _, _, E0o, gap = O_green_exact(m, nu, nd, om_r + 0.1j, spin)
                if gap < 1e-6:
                    pytest.skip("degenerate ground state")
                assert abs(E - E0o) <= 1e-10 * max(1.0, abs(E0o))
                G = ed.ed_sym_green(s, om_r, m.ns, eta=0.1, axis=ed.ED_AXIS_REAL, spin=spin)
                assert np.max(np.abs(G - Gr)) <= 1e-8, np.max(np.abs(G - Gr))
                Gm = O_green_exact(m, nu, nd, 1j * om_m, spin)[0]
                G = ed.ed_sym_green(s, om_m, m.ns, axis=ed.ED_AXIS_MATSUBARA, spin=spin)
                assert np.max(np.abs(G - Gm)) <= 1e-8, np.max(np.abs(G - Gm))
        finally:
            ed.ed_sym_destroy(s)
    finally:
        ed.ed_cluster_destroy(hc)


def O_green_exact(m, nu, nd, z, spin):
    return OM.green_exact(m, nu, nd, np.asarray(z), spin=spin)


def test_symmetrized_green_function_3x4_matches_the_unsymmetrized_path():
    """The interacting half-filled 3x4 cluster (853,776 states): G of the A1 ground state from the
    symmetrized sectors against the library's own continued-fraction G on the full sectors
    (itself oracle-pinned), Matsubara axis."""
    h, mx, my = rect(4, 3)
    t = h
    c = {"t": t, "U": np.full(12, 4.0), "mu": 2.0, "n_up": 6, "n_dn": 6}
    hc = ed.ed_cluster_create(c, precision=ed.ED_FP64, gf_method=ed.ED_GF_CF, seed=5, tol=1e-13)
    try:
        om = (2 * np.arange(16) + 1) * np.pi / 50.0
        G_full = ed.ed_green(hc, om, 0.0, 12, spin=0, axis=ed.ED_AXIS_MATSUBARA)[1]
        ir, s, E = _ground_irrep(hc, [mx, my])
        try:
            G = ed.ed_sym_green(s, om, 12, axis=ed.ED_AXIS_MATSUBARA)
            assert np.max(np.abs(G - G_full)) <= 1e-8, np.max(np.abs(G - G_full))
        finally:
            ed.ed_sym_destroy(s)
    finally:
        ed.ed_cluster_destroy(hc)


# ---- Abelian groups with complex characters (Sec. 4.5): rotations of order 4, ring translations


def _ring(L, t1=-1.0, t2=0.0):
    t = np.zeros((L, L))
    for i in range(L):
        t[i, (i + 1) % L] = t[(i + 1) % L, i] = t1
        if t2:
            t[i, (i + 2) % L] = t[(i + 2) % L, i] = t2
    return t


def _abelian_cases():
    """(name, (t, U, mu, n_up, n_dn[, eps, theta]), generators, orders)."""
    out = []
    t = _ring(4)
    tr4 = [(i + 1) % 4 for i in range(4)]
    out.append(("ring4 C4", (t, 5.0, 2.5, 2, 2), [tr4], (4,)))
    out.append(("ring4 C4 odd filling", (t, 5.0, 2.5, 1, 2), [tr4], (4,)))
    out.append(("ring6 C6 t'", (_ring(6, -1.0, 0.3), 4.0, 2.0, 3, 2), [[(i + 1) % 6 for i in range(6)]], (6,)))
    h, _, _ = rect(2, 2)
    h[0, 3] = h[3, 0] = h[1, 2] = h[2, 1] = 0.3
    rot = [1, 3, 0, 2]  # (x, y) -> (1 - y, x) on s = x + 2 y
    out.append(("plaquette + bath C4", (h, 8.0, 4.0, 3, 3, np.full(4, -1.0), 0.5 * np.eye(4)),
                [rot + [4 + v for v in rot]], (4,)))
    t = np.zeros((8, 8))
    for x in range(4):
        t[x, (x + 1) % 4] = t[(x + 1) % 4, x] = -1.0
        t[4 + x, 4 + (x + 1) % 4] = t[4 + (x + 1) % 4, 4 + x] = -1.0
        t[x, 4 + x] = t[4 + x, x] = -0.5
    tr = [(s + 1) % 4 + 4 * (s // 4) for s in range(8)]
    leg = [(s + 4) % 8 for s in range(8)]
    out.append(("ladder 2x4 Z4 x Z2", (t, 3.0, 1.5, 3, 3), [tr, leg], (4, 2)))
    # 12-site periodic ring, the twelve momenta: sectors of about 20,000 states
    out.append(("ring12 C12", (_ring(12, -1.0, 0.2), 4.0, 2.0, 4, 4), [[(i + 1) % 12 for i in range(12)]], (12,)))
    return out


def _check_abelian_irrep(hc, m, nu, nd, gens, orders, ir):
    L = m.L
    s = ed.ed_sym_create_abelian(hc, np.array(gens), orders, ir)
    try:
        bu, bd, st = S.symmetric_basis(L, nu, nd, gens, ir, orders)
        keys, stab = ed.ed_sym_basis(s)
        okey = (bu.astype(np.uint64) << np.uint64(L)) | bd.astype(np.uint64)
        assert np.array_equal(keys, okey)
        assert np.array_equal(stab.astype(np.int64), st)
        if len(keys) == 0:
            return None
        Ho, _ = S.symmetric_hamiltonian(m, nu, nd, gens, ir, orders)
        cplx = ed.ed_sym_is_complex(s)
        assert cplx == np.iscomplexobj(Ho.data)
        Hg = _device_csr(s)
        assert np.array_equal(Hg.indptr, Ho.indptr) and np.array_equal(Hg.indices, Ho.indices)
        assert np.max(np.abs(Hg.data - Ho.data)) <= 1e-14 * max(1.0, np.max(np.abs(Ho.data)))
        rng = np.random.default_rng(len(keys))
        x = rng.standard_normal(len(keys)) + (1j * rng.standard_normal(len(keys)) if cplx else 0.0)
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        ed.ed_sym_hpsi(s, xd.data_ptr(), yd.data_ptr())
        ref = Ho @ x
        assert np.max(np.abs(yd.cpu().numpy() - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
        E, res, it, st_ = ed.ed_sym_ground_state(s)
        Eo = OM.irrep_ground_energy(Ho, m, nu, nd, gens, ir, orders=orders)
        assert abs(E - Eo) <= 1e-10 * max(1.0, abs(Eo)), (E, Eo)
        assert res <= 1e-12 * max(1.0, abs(E))
        w = ed.ed_sym_ground_vector(s)
        assert np.iscomplexobj(w) == cplx
        assert abs(np.linalg.norm(w) - 1.0) < 1e-12
        assert np.linalg.norm(Ho @ w - E * w) <= 1e-11 * max(1.0, abs(E))
        return E
    finally:
        ed.ed_sym_destroy(s)


@pytest.mark.parametrize("case", _abelian_cases(), ids=lambda c: c[0])
def test_abelian_sector_matches_oracle(case):
    """Every irrep of a group with complex characters: representatives and stabilizers bit for
    bit, the complex Hermitian matrix entry by entry, H.psi on complex device vectors, the irrep's
    ground energy and vector; the lowest irrep energy is the sector's ground energy."""
    name, params, gens, orders = case
    t, U, mu, nu, nd = params[:5]
    eps, theta = (params[5], params[6]) if len(params) > 5 else (None, None)
    hc, m = _cluster(t, U, mu, nu, nd, eps, theta)
    try:
        Es = [e for ir in S.all_irreps(len(gens), orders)
              if (e := _check_abelian_irrep(hc, m, nu, nd, gens, orders, ir)) is not None]
        E0, _, _ = OM.ground_state(m, nu, nd)
        assert abs(min(Es) - E0) <= 1e-10 * max(1.0, abs(E0))
    finally:
        ed.ed_cluster_destroy(hc)


def test_abelian_handle_with_sign_irreps_equals_the_involution_handle():
    """Orders 2 and exponents m_j = (1 - sign_j) / 2 name the same irrep as the signs."""
    h, mx, my = rect(3, 2)
    hc, m = _cluster(h, 4.0, 2.0, 3, 3)
    try:
        for signs in S.all_irreps(2):
            a = ed.ed_sym_create(hc, np.array([mx, my]), signs)
            b = ed.ed_sym_create_abelian(hc, np.array([mx, my]), (2, 2), [(1 - v) // 2 for v in signs])
            try:
                assert not ed.ed_sym_is_complex(a) and not ed.ed_sym_is_complex(b)
                for x, y in zip(ed.ed_sym_matrix(a), ed.ed_sym_matrix(b)):
                    assert np.array_equal(x, y)
            finally:
                ed.ed_sym_destroy(a)
                ed.ed_sym_destroy(b)
    finally:
        ed.ed_cluster_destroy(hc)


def test_invalid_abelian_groups_are_refused():
    t = _ring(6)
    hc, m = _cluster(t, 4.0, 2.0, 3, 3)
    tr = [(i + 1) % 6 for i in range(6)]
    inv = [(-i) % 6 for i in range(6)]
    try:
        bad = [
            ([tr], (4,), [0]),            # g^4 is not the identity
            ([tr], (6,), [6]),            # exponent out of range
            ([tr], (6,), [-1]),           # exponent out of range
            ([tr], (1,), [0]),            # order below 2
            ([tr, inv], (6, 2), [0, 0]),  # the reflection does not commute with the translation
            ([tr, [(i + 3) % 6 for i in range(6)]], (6, 2), [0, 0]),  # dependent: t^3
            ([tr, tr, tr], (6, 6, 6), [0, 0, 0]),  # more than 32 elements
        ]
        for perms, orders, ir in bad:
            with pytest.raises(ed.EDError) as e:
                ed.ed_sym_create_abelian(hc, np.array(perms), orders, ir)
            assert e.value.status == ed.ED_ERR_INVALID, (perms, orders, ir)
    finally:
        ed.ed_cluster_destroy(hc)


def _ground_irrep_abelian(hc, gens, orders):
    """The irrep holding the sector's ground state: (exponents, handle with its ground state, E)."""
    best = None
    for ir in S.all_irreps(len(gens), orders):
        s = ed.ed_sym_create_abelian(hc, np.array(gens), orders, ir)
        d, _ = ed.ed_sym_info(s)
        if d == 0:
            ed.ed_sym_destroy(s)
            continue
        E = ed.ed_sym_ground_state(s)[0]
        if best is None or E < best[2] - 1e-9:
            if best is not None:
                ed.ed_sym_destroy(best[1])
            best = (ir, s, E)
        else:
            ed.ed_sym_destroy(s)
    return best


def _abelian_gf_cases():
    """Clusters of _abelian_cases whose sector ground state is not degenerate, and a half-filled
    ladder; G is unique there."""
    keep = {"ring4 C4", "plaquette + bath C4", "ladder 2x4 Z4 x Z2"}
    out = [c for c in _abelian_cases() if c[0] in keep]
    t = _ring(6, -1.0, 0.3)
    out.append(("ring6 C6 t' 3/3", (t, 4.0, 2.0, 3, 3), [[(i + 1) % 6 for i in range(6)]], (6,)))
    lad = [c for c in _abelian_cases() if c[0] == "ladder 2x4 Z4 x Z2"][0]
    out.append(("ladder 2x4 Z4 x Z2 half filling", (lad[1][0], 3.0, 1.5, 4, 4), lad[2], lad[3]))
    # translations alone: two site orbits (the legs), so every irrep beta has two rows and the
    # off-diagonal fractions (phi_rho + phi_sigma, phi_rho + i phi_sigma) are needed
    out.append(("ladder 2x4 Z4 only", (lad[1][0], 3.0, 1.5, 3, 3), lad[2][:1], lad[3][:1]))
    out.append(("ladder 2x4 Z4 only half filling", (lad[1][0], 3.0, 1.5, 4, 4), lad[2][:1], lad[3][:1]))
    return out


@pytest.mark.parametrize("case", _abelian_gf_cases(), ids=lambda c: c[0])
def test_abelian_green_function_matches_oracle(case):
    """Sec. 4.6 with complex characters: G of the ground state from symmetrized operators of
    every irrep (complex unitary M), continued fractions in the complex N +- 1 irrep sectors
    (alpha + beta for c+, alpha - beta for c), off-diagonal terms from the fractions of
    phi_rho + phi_sigma and phi_rho + i phi_sigma, against the exact Lehmann sum of the
    unsymmetrized sectors (real axis, eta = 0.1, and Matsubara axis, beta = 50), both spins."""
    name, params, gens, orders = case
    t, U, mu, nu, nd = params[:5]
    eps, theta = (params[5], params[6]) if len(params) > 5 else (None, None)
    hc, m = _cluster(t, U, mu, nu, nd, eps, theta)
    try:
        ir, s, E = _ground_irrep_abelian(hc, gens, orders)
        try:
            om_r = np.linspace(-8.0, 8.0, 48)
            om_m = (2 * np.arange(24) + 1) * np.pi / 50.0
            for spin in (0, 1):
                Gr, _, _, E0o, gap = O_green_exact(m, nu, nd, om_r + 0.1j, spin)
                assert gap > 1e-6, "the cases are chosen with a non-degenerate ground state"
                assert abs(E - E0o) <= 1e-10 * max(1.0, abs(E0o))
                G = ed.ed_sym_green(s, om_r, m.ns, eta=0.1, axis=ed.ED_AXIS_REAL, spin=spin)
                assert np.max(np.abs(G - Gr)) <= 1e-8, np.max(np.abs(G - Gr))
                Gm = O_green_exact(m, nu, nd, 1j * om_m, spin)[0]
                G = ed.ed_sym_green(s, om_m, m.ns, axis=ed.ED_AXIS_MATSUBARA, spin=spin)
                assert np.max(np.abs(G - Gm)) <= 1e-8, np.max(np.abs(G - Gm))
        finally:
            ed.ed_sym_destroy(s)
    finally:
        ed.ed_cluster_destroy(hc)
