"""FP64 CPU oracle for cluster symmetries (Sec. 4.5): the Hamiltonian of one irreducible
representation of an Abelian symmetry group of the cluster, in the basis of symmetrized states.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and nothing in the product package.

Scope: groups generated by commuting involutions of the orbitals (mirrors, two-fold rotations,
half translations of a periodic cluster), so every element is its own inverse and every
irreducible representation has characters +-1 (Sec. 4.5 restricts to Abelian groups with
one-dimensional representations).  An irrep is named by the signs ``s_k`` it gives the
generators; the element ``g = prod_{k in mask} g_k`` then has character ``prod_{k in mask} s_k``.

Construction (Sec. 4.5, following the text step by step):

* A group element acts on the orbitals by a permutation ``p`` (both spins alike), so
  ``g |b> = phi_g(b) |g b>`` where ``g b`` moves the occupation of orbital ``i`` to ``p(i)`` and
  ``phi_g(b)`` is the sign of the permutation that brings the moved creation operators back to
  the canonical order (all up orbitals ascending, then all down orbitals ascending).
* Every binary state ``b = (b_up, b_dn)`` generates an orbit; its representative is the member
  with the smallest key ``b_up * 2**L + b_dn`` (the smallest binary representation, up label
  first as in ``psi[u, d]``).
* The symmetrized state of a representative ``r`` is the projection
  ``|psi(r)> ~ sum_g chi_g g |r>``; it vanishes unless ``chi_g phi_g(r) = 1`` for every ``g`` of
  the stabilizer ``S_r = {g : g r = r}``, and then its norm squared is ``|G| |S_r|``.
* Matrix elements (Eq. matrixElement, written for normalized states): applying each term of H
  to ``r1`` gives binary states ``b_k`` with amplitudes ``h_k``; if ``g_k b_k = r_k`` (its
  representative) then ``P |b_k> = phi_{g_k}(b_k) chi_{g_k} P |r_k>`` and

      <psi(r2)| H |psi(r1)> = sum_{k : r_k = r2} h_k phi_{g_k}(b_k) chi_{g_k} sqrt(|S_r2| / |S_r1|).

  The column of ``r1`` is accumulated first, so the cancellations between terms mentioned in
  Sec. 4.5 take place before it is stored.

Parity status: pinned in tests/test_symmetry_oracle_pins.py by the dimensions and by the counts
of every matrix-element magnitude of Table 1 (nearest-neighbour hopping on the half-filled 3x4
cluster, group C2v), by the spectrum of the unsymmetrized sector being the union of the irrep
spectra (several clusters and groups), and by the dimension formula (1/|G|) sum_g chi_g Tr(g).
"""

from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .ed_oracle import Model, _between_mask, sector_basis, popcount


def group_elements(gens, n_orb):
    """All elements of the group generated by ``gens`` (lists of n_orb orbital images), as
    (mask, permutation) pairs; the generators must be commuting, independent involutions."""
    gens = [np.asarray(g, dtype=np.int64) for g in gens]
    for g in gens:
        if sorted(g.tolist()) != list(range(n_orb)):
            raise ValueError("a generator is not a permutation of the orbitals")
        if not np.array_equal(g[g], np.arange(n_orb)):
            raise ValueError("a generator is not an involution")
    for g, h in itertools.combinations(gens, 2):
        if not np.array_equal(g[h], h[g]):
            raise ValueError("generators do not commute")
    out = []
    for mask in range(1 << len(gens)):
        p = np.arange(n_orb)
        for k, g in enumerate(gens):
            if mask >> k & 1:
                p = g[p]
        out.append((mask, p))
    if len({tuple(p) for _, p in out}) != len(out):
        raise ValueError("generators are not independent")
    return out


def character(mask, irrep):
    """chi_g of the element with the given generator mask in the irrep of generator signs."""
    c = 1
    for k, s in enumerate(irrep):
        if mask >> k & 1:
            c *= s
    return c


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
    g b = r (the first one in mask order among those reaching the minimum), phi_g(b) and g's mask."""
    bu = np.asarray(bu, dtype=np.uint64)
    bd = np.asarray(bd, dtype=np.uint64)
    best = None
    for mask, p in G:
        gu, gd, ph = apply_element(p, bu, bd)
        key = (gu << np.uint64(L)) | gd
        if best is None:
            best = [key, gu, gd, ph, np.full(bu.shape, mask, dtype=np.int64)]
            continue
        lt = key < best[0]
        best[0] = np.where(lt, key, best[0])
        best[1] = np.where(lt, gu, best[1])
        best[2] = np.where(lt, gd, best[2])
        best[3] = np.where(lt, ph, best[3])
        best[4] = np.where(lt, mask, best[4])
    return best[1], best[2], best[3], best[4]


def symmetric_basis(L, n_up, n_dn, gens, irrep):
    """Representatives (b_up, b_dn) of the non-vanishing symmetrized states of the irrep, in
    ascending key order, and their stabilizer sizes |S_r|."""
    G = group_elements(gens, L)
    Bu = sector_basis(L, n_up).astype(np.uint64)
    Bd = sector_basis(L, n_dn).astype(np.uint64)
    bu = np.repeat(Bu, len(Bd))
    bd = np.tile(Bd, len(Bu))
    key = (bu << np.uint64(L)) | bd
    is_rep = np.ones(key.shape, dtype=bool)
    stab = np.zeros(key.shape, dtype=np.int64)
    ok = np.ones(key.shape, dtype=bool)
    for mask, p in G:
        gu, gd, ph = apply_element(p, bu, bd)
        gkey = (gu << np.uint64(L)) | gd
        is_rep &= key <= gkey
        fixed = gkey == key
        stab += fixed
        ok &= ~fixed | (character(mask, irrep) * ph == 1)
    keep = is_rep & ok
    return bu[keep], bd[keep], stab[keep]


def irrep_dimension_formula(L, n_up, n_dn, gens, irrep):
    """dim = (1/|G|) sum_g chi_g Tr(g) over the unsymmetrized sector, Tr(g) = sum of phi_g(b)
    over the binary states that g fixes (the character formula for the multiplicity)."""
    G = group_elements(gens, L)
    Bu = sector_basis(L, n_up).astype(np.uint64)
    Bd = sector_basis(L, n_dn).astype(np.uint64)
    bu = np.repeat(Bu, len(Bd))
    bd = np.tile(Bd, len(Bu))
    tot = 0
    for mask, p in G:
        gu, gd, ph = apply_element(p, bu, bd)
        fixed = (gu == bu) & (gd == bd)
        tot += character(mask, irrep) * int(ph[fixed].sum())
    assert tot % len(G) == 0
    return tot // len(G)


def _directed_hops(h):
    n = h.shape[0]
    return [(a, b, float(h[a, b])) for a in range(n) for b in range(n) if a != b and h[a, b] != 0.0]


def symmetric_hamiltonian(model: Model, n_up, n_dn, gens, irrep):
    """H of the irrep in the orthonormal symmetrized basis (scipy CSR, rows and columns in the
    order of symmetric_basis), with the basis (b_up, b_dn, |S|)."""
    L = model.L
    G = group_elements(gens, L)
    h = model.h
    for mask, p in G:
        if not np.allclose(h[np.ix_(p, p)], h):
            raise ValueError("the one-body matrix is not invariant under the group")
        if not np.allclose(model.U[p], model.U):
            raise ValueError("the interaction is not invariant under the group")
    bu, bd, S = symmetric_basis(L, n_up, n_dn, gens, irrep)
    key = (bu << np.uint64(L)) | bd
    dim = len(key)
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
            chi = np.array([character(int(m), irrep) for m in gm], dtype=np.float64)
            coef = hab * jw * ph * chi * np.sqrt(S[pos_c] / S[src])
            rows.append(pos_c[found])
            cols.append(src[found])
            vals.append(coef[found])
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(dim, dim)).tocsr()
    H.sum_duplicates()
    H.data[np.abs(H.data) < 1e-13] = 0.0
    H.eliminate_zeros()
    return H, (bu, bd, S)


def all_irreps(n_gens):
    """Every irrep as its tuple of generator signs."""
    return list(itertools.product((1, -1), repeat=n_gens))


def irrep_spectra(model: Model, n_up, n_dn, gens):
    """Dense eigenvalues of every irrep's H (small sectors), keyed by irrep."""
    out = {}
    for ir in all_irreps(len(gens)):
        H, _ = symmetric_hamiltonian(model, n_up, n_dn, gens, ir)
        out[ir] = np.linalg.eigvalsh(H.toarray()) if H.shape[0] else np.zeros(0)
    return out


def irrep_ground_energy(model: Model, n_up, n_dn, gens, irrep, dense_limit=4000):
    """Lowest eigenvalue of the irrep's H (dense below dense_limit, else ARPACK)."""
    H, _ = symmetric_hamiltonian(model, n_up, n_dn, gens, irrep)
    if H.shape[0] == 0:
        return np.inf
    if H.shape[0] <= dense_limit:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    import scipy.sparse.linalg as sla

    return float(sla.eigsh(H, k=1, which="SA", tol=1e-14)[0][0])
