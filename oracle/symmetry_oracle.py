"""FP64 CPU oracle for cluster symmetries (Sec. 4.5): the Hamiltonian of one irreducible
representation of an Abelian symmetry group of the cluster, in the basis of symmetrized states.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and nothing in the product package.

Scope: Abelian groups (Sec. 4.5 restricts to those, whose irreducible representations are all
one-dimensional), given by commuting, independent generators g_k of orders n_k acting on the
orbitals: mirrors and two-fold rotations (n = 2), four-fold rotations, translations of a periodic
cluster.  The element g_a = prod_k g_k^{a_k} (0 <= a_k < n_k) has character
chi(g_a) = exp(2 pi i sum_k m_k a_k / n_k) in the irrep named by the integers m_k.  Without
explicit orders every generator is an involution and an irrep is named by the signs
s_k = (-1)^{m_k} it gives the generators (real characters +-1).

Construction (Sec. 4.5, following the text step by step):

* A group element acts on the orbitals by a permutation ``p`` (both spins alike), so
  ``g |b> = phi_g(b) |g b>`` where ``g b`` moves the occupation of orbital ``i`` to ``p(i)`` and
  ``phi_g(b)`` is the sign of the permutation that brings the moved creation operators back to
  the canonical order (all up orbitals ascending, then all down orbitals ascending).
* Every binary state ``b = (b_up, b_dn)`` generates an orbit; its representative is the member
  with the smallest key ``b_up * 2**L + b_dn`` (the smallest binary representation, up label
  first as in ``psi[u, d]``).
* The symmetrized state of a representative ``r`` is the projection
  ``|psi(r)> ~ P |r>, P = (1/|G|) sum_g chi_g^* g``; it vanishes unless ``chi_g = phi_g(r)`` for
  every ``g`` of the stabilizer ``S_r = {g : g r = r}``, and then ``|P r|^2 = |S_r| / |G|``.
* Matrix elements (Eq. matrixElement, written for normalized states): ``P g = chi_g P``, so if
  applying a term of H to ``r1`` gives the binary state ``b_k`` with amplitude ``h_k`` and
  ``g_k b_k = r_k`` (its representative), then ``P |b_k> = phi_{g_k}(b_k) chi_{g_k}^* P |r_k>`` and

      <psi(r2)| H |psi(r1)> = sum_{k : r_k = r2} h_k phi_{g_k}(b_k) chi_{g_k}^* sqrt(|S_r2| / |S_r1|),

  a Hermitian matrix, real when every character is.

  The column of ``r1`` is accumulated first, so the cancellations between terms mentioned in
  Sec. 4.5 take place before it is stored.

Parity status: pinned in tests/test_symmetry_oracle_pins.py by the dimensions and by the counts
of every matrix-element value of Table 1 (nearest-neighbour hopping on the half-filled 3x4
cluster, group C2v), by the spectrum of the unsymmetrized sector being the union of the irrep
spectra (clusters with real and with complex characters: C2v, inversion, C4 rotations,
translations of rings and ladders), and by the dimension formula (1/|G|) sum_g chi_g^* Tr(g).
"""

from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .ed_oracle import Model, _between_mask, sector_basis, popcount


def group_elements(gens, n_orb, orders=None):
    """All elements of the group generated by ``gens`` (lists of n_orb orbital images) with the
    given orders (None: every generator an involution), as (exponents a, permutation) pairs in
    lexicographic order of a; the generators must commute and be independent."""
    gens = [np.asarray(g, dtype=np.int64) for g in gens]
    orders = (2,) * len(gens) if orders is None else tuple(int(o) for o in orders)
    ident = np.arange(n_orb)
    for g, n in zip(gens, orders):
        if sorted(g.tolist()) != list(range(n_orb)):
            raise ValueError("a generator is not a permutation of the orbitals")
        q = ident.copy()
        for _ in range(n):
            q = g[q]
        if not np.array_equal(q, ident):
            raise ValueError("a generator is not an involution" if n == 2 else "a generator's order does not divide n")
    for g, h in itertools.combinations(gens, 2):
        if not np.array_equal(g[h], h[g]):
            raise ValueError("generators do not commute")
    out = []
    for a in itertools.product(*[range(n) for n in orders]):
        p = ident.copy()
        for g, ak in zip(gens, a):
            for _ in range(ak):
                p = g[p]
        out.append((a, p))
    if len({tuple(p) for _, p in out}) != len(out):
        raise ValueError("generators are not independent")
    return out


def character(a, irrep, orders=None):
    """chi(g_a) in the irrep: prod_k s_k^{a_k} for involution generators named by signs s_k (real),
    else exp(2 pi i sum_k m_k a_k / n_k) for the exponents m_k (complex)."""
    if orders is None:
        c = 1
        for ak, sk in zip(a, irrep):
            if ak & 1:
                c *= sk
        return c
    return np.exp(2j * np.pi * sum(mk * ak / nk for mk, ak, nk in zip(irrep, a, orders)))


def moved_bits(p, b):
    """g b for one spin string (array of uint64): orbital i's bit moves to p[i]."""
    b = np.asarray(b, dtype=np.uint64)
    out = np.zeros_like(b)
    for i, pi in enumerate(p):
        out |= ((b >> np.uint64(i)) & np.uint64(1)) << np.uint64(int(pi))
    return out


def perm_sign(p, b):
    """(-1)^(number of inversions of p among the occupied orbitals of b), per element of b:
    the sign of reordering the moved creation operators of one spin."""
    b = np.asarray(b, dtype=np.uint64)
    par = np.zeros(b.shape, dtype=np.int64)
    n = len(p)
    for i in range(n):
        bi = ((b >> np.uint64(i)) & np.uint64(1)).astype(np.int64)
        for j in range(i + 1, n):
            if p[i] > p[j]:
                par ^= bi & ((b >> np.uint64(j)) & np.uint64(1)).astype(np.int64)
    return 1 - 2 * par


def apply_element(p, bu, bd):
    """g (b_up, b_dn) and the phase phi_g(b) (the two spins reorder separately)."""
    return moved_bits(p, bu), moved_bits(p, bd), perm_sign(p, bu) * perm_sign(p, bd)


def representative(G, bu, bd, L):
    """For binary states (arrays), the orbit representative (b_up, b_dn), the element g with
    g b = r (the first one in element order among those reaching the minimum), phi_g(b) and g's
    index in G."""
    bu = np.asarray(bu, dtype=np.uint64)
    bd = np.asarray(bd, dtype=np.uint64)
    best = None
    for idx, (a, p) in enumerate(G):
        gu, gd, ph = apply_element(p, bu, bd)
        key = (gu << np.uint64(L)) | gd
        if best is None:
            best = [key, gu, gd, ph, np.full(bu.shape, idx, dtype=np.int64)]
            continue
        lt = key < best[0]
        best[0] = np.where(lt, key, best[0])
        best[1] = np.where(lt, gu, best[1])
        best[2] = np.where(lt, gd, best[2])
        best[3] = np.where(lt, ph, best[3])
        best[4] = np.where(lt, idx, best[4])
    return best[1], best[2], best[3], best[4]


def symmetric_basis(L, n_up, n_dn, gens, irrep, orders=None):
    """Representatives (b_up, b_dn) of the non-vanishing symmetrized states of the irrep, in
    ascending key order, and their stabilizer sizes |S_r|."""
    G = group_elements(gens, L, orders)
    Bu = sector_basis(L, n_up).astype(np.uint64)
    Bd = sector_basis(L, n_dn).astype(np.uint64)
    bu = np.repeat(Bu, len(Bd))
    bd = np.tile(Bd, len(Bu))
    key = (bu << np.uint64(L)) | bd
    is_rep = np.ones(key.shape, dtype=bool)
    stab = np.zeros(key.shape, dtype=np.int64)
    ok = np.ones(key.shape, dtype=bool)
    for a, p in G:
        gu, gd, ph = apply_element(p, bu, bd)
        gkey = (gu << np.uint64(L)) | gd
        is_rep &= key <= gkey
        fixed = gkey == key
        stab += fixed
        ok &= ~fixed | (np.abs(character(a, irrep, orders) - ph) < 1e-9)
    keep = is_rep & ok
    return bu[keep], bd[keep], stab[keep]


def irrep_dimension_formula(L, n_up, n_dn, gens, irrep, orders=None):
    """dim = (1/|G|) sum_g chi_g^* Tr(g) over the unsymmetrized sector, Tr(g) = sum of phi_g(b)
    over the binary states that g fixes (the character formula for the multiplicity)."""
    G = group_elements(gens, L, orders)
    Bu = sector_basis(L, n_up).astype(np.uint64)
    Bd = sector_basis(L, n_dn).astype(np.uint64)
    bu = np.repeat(Bu, len(Bd))
    bd = np.tile(Bd, len(Bu))
    tot = 0
    for a, p in G:
        gu, gd, ph = apply_element(p, bu, bd)
        fixed = (gu == bu) & (gd == bd)
        tot += np.conj(character(a, irrep, orders)) * int(ph[fixed].sum())
    d = tot / len(G)
    assert abs(d - round(d.real)) < 1e-9
    return int(round(d.real))


def _directed_hops(h):
    n = h.shape[0]
    return [(a, b, float(h[a, b])) for a in range(n) for b in range(n) if a != b and h[a, b] != 0.0]


def symmetric_hamiltonian(model: Model, n_up, n_dn, gens, irrep, orders=None):
    """H of the irrep in the orthonormal symmetrized basis (scipy CSR, rows and columns in the
    order of symmetric_basis; complex Hermitian when a character is complex), with the basis
    (b_up, b_dn, |S|)."""
    L = model.L
    G = group_elements(gens, L, orders)
    h = model.h
    for a_, p in G:
        if not np.allclose(h[np.ix_(p, p)], h):
            raise ValueError("the one-body matrix is not invariant under the group")
        if not np.allclose(model.U[p], model.U):
            raise ValueError("the interaction is not invariant under the group")
    bu, bd, S = symmetric_basis(L, n_up, n_dn, gens, irrep, orders)
    key = (bu << np.uint64(L)) | bd
    dim = len(key)
    chis = np.array([character(a, irrep, orders) for a, _ in G])
    cplx = np.iscomplexobj(chis) and np.max(np.abs(np.imag(chis))) > 1e-12
    rows, cols, vals = [], [], []
    # diagonal: one-body diagonal and Hubbard U (the same for every member of an orbit)
    diag = np.zeros(dim)
    for a in range(L):
        na = ((bu >> np.uint64(a)) & np.uint64(1)).astype(np.float64) + ((bd >> np.uint64(a)) & np.uint64(1)).astype(np.float64)
        diag += h[a, a] * na
    for i, Ui in enumerate(model.U):
        if Ui != 0.0:
            diag += Ui * (((bu >> np.uint64(i)) & (bd >> np.uint64(i)) & np.uint64(1)).astype(np.float64))
    rows.append(np.arange(dim))
    cols.append(np.arange(dim))
    vals.append(diag)
    idx_all = np.arange(dim)
    for a, b, hab in _directed_hops(h):
        between = np.uint64(_between_mask(a, b))
        for spin in (0, 1):
            bs = bu if spin == 0 else bd
            can = (((bs >> np.uint64(b)) & np.uint64(1)) == 1) & (((bs >> np.uint64(a)) & np.uint64(1)) == 0)
            if not can.any():
                continue
            src = idx_all[can]
            flip = np.uint64((1 << a) | (1 << b))
            nu = bu[can] ^ flip if spin == 0 else bu[can]
            nd = bd[can] ^ flip if spin == 1 else bd[can]
            jw = 1.0 - 2.0 * (popcount(bs[can] & between) & 1)
            ru, rd, ph, gm = representative(G, nu, nd, L)
            rkey = (ru << np.uint64(L)) | rd
            pos = np.searchsorted(key, rkey)
            pos_c = np.minimum(pos, dim - 1)
            found = (pos < dim) & (key[pos_c] == rkey)
            chi = np.conj(chis[gm]) if cplx else np.real(chis[gm]).astype(np.float64)
            coef = hab * jw * ph * chi * np.sqrt(S[pos_c] / S[src])
            rows.append(pos_c[found])
            cols.append(src[found])
            vals.append(coef[found])
    dt = np.complex128 if cplx else np.float64
    H = sp.coo_matrix((np.concatenate([np.asarray(v, dtype=dt) for v in vals]),
                       (np.concatenate(rows), np.concatenate(cols))), shape=(dim, dim)).tocsr()
    H.sum_duplicates()
    H.data[np.abs(H.data) < 1e-13] = 0.0
    H.eliminate_zeros()
    return H, (bu, bd, S)


def embed(vec, basis, L, n_up, n_dn, gens, irrep, orders=None):
    """The unsymmetrized sector vector psi[u, d] of sum_r vec[r] |psi(r)>, from the definition
    |psi(r)> = sqrt(|G| / |S_r|) (1/|G|) sum_g chi_g^* phi_g(r) |g r>."""
    bu, bd, st = basis
    G = group_elements(gens, L, orders)
    Bu = sector_basis(L, n_up).astype(np.uint64)
    Bd = sector_basis(L, n_dn).astype(np.uint64)
    out = np.zeros((len(Bu), len(Bd)), dtype=np.complex128)
    pref = np.sqrt(len(G) / st.astype(np.float64)) / len(G)
    for a, p in G:
        gu, gd, ph = apply_element(p, bu, bd)
        iu = np.searchsorted(Bu, gu)
        idd = np.searchsorted(Bd, gd)
        np.add.at(out, (iu, idd), np.conj(character(a, irrep, orders)) * ph * pref * np.asarray(vec))
    return out


def apply_group_element(psi, p, L, n_up, n_dn):
    """g psi for a sector vector psi[u, d]: g|b> = phi_g(b) |g b>."""
    Bu = sector_basis(L, n_up).astype(np.uint64)
    Bd = sector_basis(L, n_dn).astype(np.uint64)
    bu = np.repeat(Bu, len(Bd))
    bd = np.tile(Bd, len(Bu))
    gu, gd, ph = apply_element(p, bu, bd)
    out = np.zeros_like(psi)
    out[np.searchsorted(Bu, gu), np.searchsorted(Bd, gd)] = ph * psi.reshape(-1)
    return out


def all_irreps(n_gens, orders=None):
    """Every irrep: tuples of generator signs for involution generators (orders None), else
    tuples of exponents m_k, 0 <= m_k < n_k."""
    if orders is None:
        return list(itertools.product((1, -1), repeat=n_gens))
    return list(itertools.product(*[range(int(n)) for n in orders]))


def irrep_spectra(model: Model, n_up, n_dn, gens, orders=None):
    """Dense eigenvalues of every irrep's H (small sectors), keyed by irrep."""
    out = {}
    for ir in all_irreps(len(gens), orders):
        H, _ = symmetric_hamiltonian(model, n_up, n_dn, gens, ir, orders)
        out[ir] = np.linalg.eigvalsh(H.toarray()) if H.shape[0] else np.zeros(0)
    return out


def irrep_ground_energy(model: Model, n_up, n_dn, gens, irrep, dense_limit=4000, orders=None):
    """Lowest eigenvalue of the irrep's H (dense below dense_limit, else ARPACK)."""
    H, _ = symmetric_hamiltonian(model, n_up, n_dn, gens, irrep, orders)
    if H.shape[0] == 0:
        return np.inf
    if H.shape[0] <= dense_limit:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    import scipy.sparse.linalg as sla

    return float(sla.eigsh(H, k=1, which="SA", tol=1e-14)[0][0])
