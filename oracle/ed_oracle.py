"""FP64 CPU oracle: exact diagonalization of a Hubbard-like cluster in a fixed (N_up, N_dn) sector.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py``; never by the product package, and it imports nothing from it.

Model (Eq. Hubbard, Sec. 1, with the bath terms of Eq. cdmft1, Sec. 6)::

    H = sum_{a,b,s} h_ab c+_{a s} c_{b s} + sum_{i in cluster sites} U_i n_{i up} n_{i dn}

over L = n_sites + n_bath orbitals (cluster sites first, then bath orbitals), with the
one-body matrix ``h`` built by :func:`one_body_matrix`:

    h[i, j]           = t[i, j]              cluster sites, i != j
    h[i, i]           = t[i, i] - mu         the chemical potential acts on cluster sites only
    h[i, ns + a]      = theta[i, a]          (and its transpose) cluster-bath hybridization
    h[ns + a, ns + a] = eps[a]               bath energies are absolute

Basis convention (Sec. 4.1, Eq. basis): bit ``a`` of ``b_s`` is the occupation of orbital
``a`` with spin ``s``; the creation operators of a basis state are ordered all-up (orbital
0 first) then all-down, so the global bit string is ``b = b_up + 2**L b_dn``.  Each spin's
states are labelled by ascending integer value.  State vectors are arrays ``psi[u, d]``
(up label slow, down label fast).

Parity status of each function (what pins it, in tests/test_oracle_pins.py):

* sector_basis, hopping_matrix, hop_entries, interaction_diagonal: pinned (binomial
  dimension of Eq. Hilbert1; combinatorial-number-system rank; the worked sign example of
  Sec. 4.1; closed-form nnz; element-wise agreement with the Jordan-Wigner engine).
* jw_hamiltonian_dense, sector_hamiltonian, apply_h: pinned (two-site closed form; U = 0
  free fermions; atomic limit; Hermiticity; JW vs factorized agreement).
* ground_state: pinned (same closed forms, dense vs sparse eigensolver on > 1 size).
* apply_cdag / apply_c, green_exact: pinned (U = 0 resolvent Eq. G0; sum rule Eq. norm;
  first-moment rule; G_ij = G_ji; z G(z) -> 1; one-site atomic closed form).
* lanczos_coefficients, cf_green, green_cf: pinned (agreement with green_exact on
  interacting clusters; sum rules b0e^2 + b0h^2 = 1).
* band_lanczos_lehmann, green_band: pinned (Q Q^T = 1; agreement with green_exact).
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "popcount", "one_body_matrix", "Model", "sector_basis", "basis_index",
    "hopping_matrix", "hop_entries", "interaction_diagonal", "sector_hamiltonian",
    "apply_h", "apply_h_rows", "row_tables", "apply_h_rows_tables", "apply_h_sampled",
    "jw_hamiltonian_dense", "ground_state",
    "apply_cdag", "apply_c", "density", "green_exact", "lanczos_coefficients",
    "cf_green", "green_cf", "band_lanczos_lehmann", "lehmann_green", "green_band",
    "frequency_grid", "low_states", "mixed_weights", "green_mixed",
]

_POP8 = np.array([bin(i).count("1") for i in range(256)], dtype=np.int64)


def popcount(x):
    """Number of set bits of each element of an unsigned integer array (byte table)."""
    x = np.asarray(x, dtype=np.uint64)
    c = np.zeros(x.shape, dtype=np.int64)
    for k in range(0, 64, 8):
        c += _POP8[((x >> np.uint64(k)) & np.uint64(255)).astype(np.int64)]
    return c


def one_body_matrix(t, mu, eps=None, theta=None):
    """One-body matrix h of Eq. Hubbard (+t convention) plus the bath terms of Eq. cdmft1."""
    t = np.asarray(t, dtype=np.float64)
    ns = t.shape[0]
    eps = np.zeros(0) if eps is None else np.asarray(eps, dtype=np.float64).ravel()
    nb = eps.shape[0]
    theta = np.zeros((ns, nb)) if theta is None else np.asarray(theta, dtype=np.float64).reshape(ns, nb)
    L = ns + nb
    h = np.zeros((L, L))
    h[:ns, :ns] = t
    h[np.arange(ns), np.arange(ns)] -= mu
    h[:ns, ns:] = theta
    h[ns:, :ns] = theta.T
    h[ns + np.arange(nb), ns + np.arange(nb)] = eps
    return h


class Model:
    """A cluster (sites + bath) in the form of Eq. cdmft1: one-body matrix h and on-site U."""

    def __init__(self, t, U, mu, eps=None, theta=None):
        self.h = one_body_matrix(t, mu, eps, theta)
        self.ns = int(np.asarray(t).shape[0])
        self.L = int(self.h.shape[0])
        self.U = np.zeros(self.L)
        self.U[: self.ns] = np.broadcast_to(np.asarray(U, dtype=np.float64), (self.ns,))


# ---------------------------------------------------------------------------------------
# Sec. 4.1: coding of the basis states
# ---------------------------------------------------------------------------------------

def sector_basis(L, N):
    """All L-bit strings with N set bits, in ascending integer order (Sec. 4.1, Eq. Hilbert1).

    Its length is d(N) = L! / (N! (L-N)!).  The position of a string in this array is its
    label I(b); the array itself is the inverse table B(i) of Sec. 4.1.
    """
    if N < 0 or N > L:
        return np.zeros(0, dtype=np.uint64)
    b = np.arange(1 << L, dtype=np.uint64)
    return b[popcount(b) == N]


def basis_index(B, b):
    """Label I(b) of bit strings b in the sorted table B (the two-way look-up of Sec. 4.1)."""
    idx = np.searchsorted(B, np.asarray(b, dtype=np.uint64))
    if np.any(idx >= len(B)) or np.any(B[np.minimum(idx, len(B) - 1)] != b):
        raise KeyError("bit string not in sector")
    return idx


def _between_mask(a, b):
    """Bits strictly between orbitals a and b."""
    lo, hi = min(a, b), max(a, b)
    return ((1 << hi) - 1) ^ ((1 << (lo + 1)) - 1)


def hop_entries(h, N):
    """Off-diagonal elements of K = sum_{a != b} h_ab c+_a c_b for one spin (Sec. 4.1).

    Two states are connected when their bit strings differ at orbitals a and b; the element
    is (-1)^{M_ab} h_ab with M_ab the number of occupied orbitals strictly between a and b.
    Returns int arrays (row, col, a, b, sign): K[row, col] += sign * h[a, b], where col is the
    label of the source state (b occupied, a empty) and row the label of the target state.
    """
    L = h.shape[0]
    B = sector_basis(L, N)
    out = [[], [], [], [], []]
    for b in range(L):
        for a in range(L):
            if a == b or h[a, b] == 0.0:
                continue
            sel = (((B >> np.uint64(b)) & np.uint64(1)) == 1) & (((B >> np.uint64(a)) & np.uint64(1)) == 0)
            src = np.nonzero(sel)[0]
            if len(src) == 0:
                continue
            new = B[src] ^ np.uint64((1 << a) | (1 << b))
            M = popcount(B[src] & np.uint64(_between_mask(a, b)))
            out[0].append(basis_index(B, new))
            out[1].append(src)
            out[2].append(np.full(len(src), a))
            out[3].append(np.full(len(src), b))
            out[4].append(1 - 2 * (M % 2))
    if not out[0]:
        return tuple(np.zeros(0, dtype=np.int64) for _ in range(5))
    return tuple(np.concatenate(c).astype(np.int64) for c in out)


def hopping_matrix(h, N):
    """Sparse K_s = sum_{a,b} h_ab c+_a c_b in the N-particle basis of one spin (Eq. factorized).

    Includes the diagonal one-body terms h_aa n_a.
    """
    L = h.shape[0]
    B = sector_basis(L, N)
    d = len(B)
    row, col, a, b, sign = hop_entries(h, N)
    vals = sign * h[a, b]
    occ = ((B[:, None] >> np.arange(L, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.float64)
    diag = occ @ np.diag(h)
    K = sp.csr_matrix((vals, (row, col)), shape=(d, d)) + sp.diags(diag)
    return K.tocsr()


def interaction_diagonal(model, B_up, B_dn):
    """V_int[u, d] = sum_i U_i n_{i up} n_{i dn}: popcount of b_up & b_dn weighted by U (Sec. 4.1)."""
    V = np.zeros((len(B_up), len(B_dn)))
    for i in range(model.L):
        if model.U[i] == 0.0:
            continue
        nu = ((B_up >> np.uint64(i)) & np.uint64(1)).astype(np.float64)
        nd = ((B_dn >> np.uint64(i)) & np.uint64(1)).astype(np.float64)
        V += model.U[i] * np.outer(nu, nd)
    return V


class SectorOperator:
    """H restricted to sector (N_up, N_dn) in factorized form (Eq. factorized)."""

    def __init__(self, model, n_up, n_dn):
        self.model = model
        self.n_up, self.n_dn = n_up, n_dn
        self.B_up = sector_basis(model.L, n_up)
        self.B_dn = sector_basis(model.L, n_dn)
        self.K_up = hopping_matrix(model.h, n_up)
        self.K_dn = hopping_matrix(model.h, n_dn)
        self.V = interaction_diagonal(model, self.B_up, self.B_dn)
        self.shape2 = (len(self.B_up), len(self.B_dn))
        self.dim = self.shape2[0] * self.shape2[1]

    def matvec(self, x):
        """y = (K_up x 1 + 1 x K_dn + V_int) x for a flat vector x in psi[u, d] order."""
        X = np.asarray(x).reshape(self.shape2)
        Y = self.K_up @ X + (self.K_dn @ X.T).T + self.V * X
        return Y.reshape(-1)

    def sparse(self):
        du, dd = self.shape2
        H = sp.kron(self.K_up, sp.identity(dd)) + sp.kron(sp.identity(du), self.K_dn)
        return (H + sp.diags(self.V.reshape(-1))).tocsr()

    def linear_operator(self):
        return spla.LinearOperator((self.dim, self.dim), matvec=self.matvec, dtype=np.float64)


def sector_hamiltonian(model, n_up, n_dn):
    """SectorOperator of Eq. factorized for the sector (n_up, n_dn)."""
    return SectorOperator(model, n_up, n_dn)


def apply_h(op, psi):
    """H psi for psi[u, d] (2-D array) using the factorized form of Eq. factorized."""
    return op.matvec(np.asarray(psi).reshape(-1)).reshape(op.shape2)


def row_tables(model, n_up, n_dn, rows):
    """The pieces of Eq. factorized that rows y[rows, :] of y = H psi need: the rows of K_up, all
    of K_dn and the rows of the interaction diagonal."""
    rows = np.asarray(rows)
    B_up = sector_basis(model.L, n_up)
    B_dn = sector_basis(model.L, n_dn)
    K_up = hopping_matrix(model.h, n_up)
    K_dn = hopping_matrix(model.h, n_dn)
    return K_up[rows], K_dn, interaction_diagonal(model, B_up[rows], B_dn)


def apply_h_rows_tables(tables, psi, rows):
    """y[rows, :] = sum_u' K_up[u, u'] psi[u', :] + psi[u, :] K_dn^T + V_int[u, :] * psi[u, :]
    (Eq. factorized) from the pieces of row_tables."""
    K_up_rows, K_dn, V = tables
    rows = np.asarray(rows)
    return K_up_rows @ psi + (K_dn @ psi[rows].T).T + V * psi[rows]


def apply_h_rows(model, n_up, n_dn, psi, rows):
    """Rows y[rows, :] of y = H psi from Eq. factorized, without building the full operator."""
    return apply_h_rows_tables(row_tables(model, n_up, n_dn, rows), psi, rows)


def apply_h_sampled(op, psi, us, ds):
    """Selected elements y[u, d] of y = H psi, each computed from its own row of K_up and K_dn."""
    us = np.asarray(us)
    ds = np.asarray(ds)
    out = np.empty(len(us))
    Ku, Kd = op.K_up, op.K_dn
    for n, (u, d) in enumerate(zip(us, ds)):
        s = op.V[u, d] * psi[u, d]
        lo, hi = Ku.indptr[u], Ku.indptr[u + 1]
        s += np.dot(Ku.data[lo:hi], psi[Ku.indices[lo:hi], d])
        lo, hi = Kd.indptr[d], Kd.indptr[d + 1]
        s += np.dot(Kd.data[lo:hi], psi[u, Kd.indices[lo:hi]])
        out[n] = s
    return out


# ---------------------------------------------------------------------------------------
# Independent Jordan-Wigner engine (global fermion ordering of Eq. basis)
# ---------------------------------------------------------------------------------------

def _jw_apply(ops, state):
    """Apply a product of fermion operators (rightmost acts first) to a global bit string.

    ``ops`` is a list of (kind, mode) with kind '+' (create) or '-' (annihilate).  Mode m
    anticommutes past every occupied mode with a smaller index (ordering of Eq. basis).
    Returns (sign, new_state), or (0, None) when the result vanishes.
    """
    sign = 1
    for kind, m in reversed(ops):
        occ = (state >> m) & 1
        if bin(state & ((1 << m) - 1)).count("1") & 1:
            sign = -sign
        if kind == "+":
            if occ:
                return 0, None
            state |= 1 << m
        else:
            if not occ:
                return 0, None
            state &= ~(1 << m)
    return sign, state


def jw_hamiltonian_dense(model, n_up, n_dn):
    """Dense H in sector (n_up, n_dn) built term by term with the Jordan-Wigner engine.

    Modes: orbital a with spin up is mode a, with spin down mode L + a (b = b_up + 2^L b_dn).
    Rows/columns are ordered psi[u, d] (flat index u * d_dn + d).  Small clusters only.
    """
    L = model.L
    B_up = [int(x) for x in sector_basis(L, n_up)]
    B_dn = [int(x) for x in sector_basis(L, n_dn)]
    states = [bu | (bd << L) for bu in B_up for bd in B_dn]
    index = {s: n for n, s in enumerate(states)}
    terms = []
    for s in (0, 1):
        for a in range(L):
            for b in range(L):
                if model.h[a, b] != 0.0:
                    terms.append((model.h[a, b], [("+", a + s * L), ("-", b + s * L)]))
    for i in range(L):
        if model.U[i] != 0.0:
            terms.append((model.U[i], [("+", i), ("-", i), ("+", i + L), ("-", i + L)]))
    H = np.zeros((len(states), len(states)))
    for col, st in enumerate(states):
        for coef, ops in terms:
            sg, new = _jw_apply(ops, st)
            if sg:
                H[index[new], col] += sg * coef
    return H


# ---------------------------------------------------------------------------------------
# Sec. 4.2: ground state (the plain definition: lowest eigenpair of H in the sector)
# ---------------------------------------------------------------------------------------

def ground_state(op, dense_limit=6000, k=2, tol=1e-14):
    """Lowest eigenvalue E0, eigenvector Omega[u, d] (unit norm) and gap E1 - E0 of H.

    Dense LAPACK (numpy.linalg.eigh) up to ``dense_limit`` states, else ARPACK (eigsh) with
    relative tolerance ``tol`` on the Ritz pairs (the eigenvalue error is of order tol^2 |E|
    for a Hermitian operator, so 1e-12 is ample for a 1e-10 check on E0).
    """
    if op.dim <= dense_limit:
        w, V = np.linalg.eigh(op.sparse().toarray())
        gap = w[1] - w[0] if len(w) > 1 else np.inf
        return w[0], V[:, 0].reshape(op.shape2), gap
    v0 = np.cos(np.arange(op.dim) * 0.7) + 1.0
    w, V = spla.eigsh(op.linear_operator(), k=k, which="SA", tol=tol, v0=v0, ncv=max(20, 2 * k + 1))
    order = np.argsort(w)
    w, V = w[order], V[:, order]
    return w[0], V[:, 0].reshape(op.shape2), (w[1] - w[0]) if k > 1 else np.inf


# ---------------------------------------------------------------------------------------
# Creation / annihilation operators (sector change N -> N +- 1, Sec. 4.3)
# ---------------------------------------------------------------------------------------

def apply_cdag(model, n_up, n_dn, psi, i, spin=0):
    """c+_{i s} psi: maps sector (n_up, n_dn) to (n_up + 1, n_dn) (spin 0) or (n_up, n_dn + 1).

    The sign is the parity of occupied modes preceding mode i in the ordering of Eq. basis;
    for a down-spin operator that includes every up electron.
    """
    L = model.L
    B_up, B_dn = sector_basis(L, n_up), sector_basis(L, n_dn)
    if spin == 0:
        Bn = sector_basis(L, n_up + 1)
        out = np.zeros((len(Bn), len(B_dn)))
        for u, b in enumerate(B_up):
            b = int(b)
            if (b >> i) & 1:
                continue
            sg = -1.0 if bin(b & ((1 << i) - 1)).count("1") & 1 else 1.0
            out[basis_index(Bn, b | (1 << i))] += sg * psi[u, :]
        return out
    Bn = sector_basis(L, n_dn + 1)
    out = np.zeros((len(B_up), len(Bn)))
    for dd, b in enumerate(B_dn):
        b = int(b)
        if (b >> i) & 1:
            continue
        sg = -1.0 if (n_up + bin(b & ((1 << i) - 1)).count("1")) & 1 else 1.0
        out[:, basis_index(Bn, b | (1 << i))] += sg * psi[:, dd]
    return out


def apply_c(model, n_up, n_dn, psi, i, spin=0):
    """c_{i s} psi: maps sector (n_up, n_dn) to (n_up - 1, n_dn) (spin 0) or (n_up, n_dn - 1)."""
    L = model.L
    B_up, B_dn = sector_basis(L, n_up), sector_basis(L, n_dn)
    if spin == 0:
        Bn = sector_basis(L, n_up - 1)
        out = np.zeros((len(Bn), len(B_dn)))
        for u, b in enumerate(B_up):
            b = int(b)
            if not (b >> i) & 1:
                continue
            sg = -1.0 if bin(b & ((1 << i) - 1)).count("1") & 1 else 1.0
            out[basis_index(Bn, b & ~(1 << i))] += sg * psi[u, :]
        return out
    Bn = sector_basis(L, n_dn - 1)
    out = np.zeros((len(B_up), len(Bn)))
    for dd, b in enumerate(B_dn):
        b = int(b)
        if not (b >> i) & 1:
            continue
        sg = -1.0 if (n_up + bin(b & ((1 << i) - 1)).count("1")) & 1 else 1.0
        out[:, basis_index(Bn, b & ~(1 << i))] += sg * psi[:, dd]
    return out


def density(model, n_up, n_dn, psi, spin):
    """<n_{i s}> for every orbital i, read directly from the amplitudes psi[u, d]."""
    B = sector_basis(model.L, n_up if spin == 0 else n_dn)
    w = (np.abs(psi) ** 2).sum(axis=1 if spin == 0 else 0)
    occ = ((B[:, None] >> np.arange(model.L, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.float64)
    return w @ occ


# ---------------------------------------------------------------------------------------
# Green function: Eq. GF1 / Eq. green, Lehmann form Eq. spectral1
# ---------------------------------------------------------------------------------------

def frequency_grid(n, lo=-8.0, hi=8.0):
    """omega_k = lo + (hi - lo) k / (n - 1), k = 0 .. n-1 (end points included)."""
    return lo + (hi - lo) * np.arange(n) / (n - 1)


def lehmann_green(Q, w, z):
    """G_ij(z) = sum_r Q[i, r] Q[j, r] / (z - w_r) (Eq. spectral1, real Q). Shape (nz, p, p)."""
    z = np.asarray(z, dtype=np.complex128).ravel()
    R = 1.0 / (z[:, None] - np.asarray(w)[None, :])
    return np.einsum("ir,zr,jr->zij", Q, R, Q)


def green_exact(model, n_up, n_dn, z, spin=0, orbitals=None, dense_limit=6000, state=None):
    """Exact G_ij(z) by full diagonalization of the N +- 1 sectors (Eqs. green, spectral1).

    Returns (G[nz, p, p], Q[p, R], w[R], E0, gap) with the electron and hole poles
    concatenated: electron poles w_r = E_r - E0, hole poles w_r = E0 - E_r (Eq. spectral1).
    ``state = (E, psi)`` takes that eigenpair of the sector in place of the ground state (the
    Green function of one of the low-lying states of a mixed state; gap is then returned as nan).
    """
    orbitals = list(range(model.ns)) if orbitals is None else list(orbitals)
    op = sector_hamiltonian(model, n_up, n_dn)
    if state is None:
        E0, Om, gap = ground_state(op, dense_limit=dense_limit)
    else:
        E0, Om, gap = float(state[0]), np.asarray(state[1]).reshape(op.shape2), float("nan")
    Qs, ws = [], []
    for kind in ("e", "h"):
        nu = n_up + (1 if kind == "e" else -1) * (spin == 0)
        nd = n_dn + (1 if kind == "e" else -1) * (spin == 1)
        if nu < 0 or nd < 0 or nu > model.L or nd > model.L:
            continue
        opx = sector_hamiltonian(model, nu, nd)
        if opx.dim == 0:
            continue
        wx, Vx = np.linalg.eigh(opx.sparse().toarray())
        f = apply_cdag if kind == "e" else apply_c
        Phi = np.stack([f(model, n_up, n_dn, Om, i, spin).reshape(-1) for i in orbitals], axis=1)
        Qs.append((Vx.T @ Phi).T)
        ws.append(wx - E0 if kind == "e" else E0 - wx)
    Q = np.concatenate(Qs, axis=1)
    w = np.concatenate(ws)
    return lehmann_green(Q, w, z), Q, w, E0, gap


def lanczos_coefficients(matvec, phi, max_steps, btol=1e-10, reorth=True):
    """Lanczos recursion of Eq. LanczosRecursion started from phi (Sec. 4.3).

    Written with normalized vectors |n> = phi_n / ||phi_n||, which is the same recursion
    without the overflow of the unnormalized form.  Returns (a[M], bsq[M]) with
    bsq[0] = b_0^2 = <phi|phi> and bsq[n] = b_n^2 for n >= 1.  The recursion stops when
    b_n < btol * b_0 (invariant subspace) or after max_steps levels.  ``reorth`` orthogonalizes
    each new vector against all previous ones (full reorthogonalization, twice).
    """
    phi = np.asarray(phi, dtype=np.float64).ravel()
    b0sq = float(phi @ phi)
    if b0sq == 0.0:
        return np.zeros(0), np.zeros(0)
    b0 = math.sqrt(b0sq)
    v = phi / b0
    v_prev = np.zeros_like(v)
    b = 0.0
    a_list, bsq_list = [], [b0sq]
    basis = [v] if reorth else None
    for n in range(max_steps):
        w = matvec(v)
        a = float(v @ w)
        w = w - a * v - b * v_prev
        if reorth:
            for _ in range(2):
                for u in basis:
                    w -= (u @ w) * u
        a_list.append(a)
        bn = float(np.linalg.norm(w))
        if n == max_steps - 1 or bn < btol * b0:
            break
        bsq_list.append(bn * bn)
        v_prev, v, b = v, w / bn, bn
        if reorth:
            basis.append(v)
    return np.array(a_list), np.array(bsq_list)


def cf_green(a, bsq, z, E0, kind):
    """Continued fraction of Eq. jacobi with the ground-energy shift of Eq. green.

    electron: b0^2 / (z - (a0 - E0) - b1^2 / (z - (a1 - E0) - ...))
    hole:     b0^2 / (z + (a0 - E0) - b1^2 / (z + (a1 - E0) - ...))
    evaluated bottom-up, truncated at the last level.
    """
    z = np.asarray(z, dtype=np.complex128)
    M = len(a)
    if M == 0:
        return np.zeros_like(z)
    sh = (np.asarray(a) - E0) if kind == "e" else -(np.asarray(a) - E0)
    den = z - sh[M - 1]
    for n in range(M - 2, -1, -1):
        den = z - sh[n] - bsq[n + 1] / den
    return bsq[0] / den


def green_cf(model, n_up, n_dn, z, spin=0, orbitals=None, max_steps=400, btol=1e-10, reorth=True,
             ground=None):
    """G_ij(z) from continued fractions (Sec. 4.3), real H: diagonal pairs from c+_i / c_i,
    off-diagonal ones from (c_i + c_j) with G_ij = (G+_ij - G_ii - G_jj) / 2.

    Returns (G[nz, p, p], coeffs) where coeffs[(kind, i, j)] = (a, bsq).
    """
    orbitals = list(range(model.ns)) if orbitals is None else list(orbitals)
    p = len(orbitals)
    op = sector_hamiltonian(model, n_up, n_dn)
    if ground is None:
        E0, Om, _ = ground_state(op)
    else:
        E0, Om = ground
    z = np.asarray(z, dtype=np.complex128).ravel()
    G = np.zeros((len(z), p, p), dtype=np.complex128)
    coeffs = {}
    for kind in ("e", "h"):
        nu = n_up + (1 if kind == "e" else -1) * (spin == 0)
        nd = n_dn + (1 if kind == "e" else -1) * (spin == 1)
        if nu < 0 or nd < 0 or nu > model.L or nd > model.L:
            continue
        opx = sector_hamiltonian(model, nu, nd)
        f = apply_cdag if kind == "e" else apply_c
        phis = [f(model, n_up, n_dn, Om, i, spin).reshape(-1) for i in orbitals]
        Gd = []
        for x in range(p):
            a, bsq = lanczos_coefficients(opx.matvec, phis[x], max_steps, btol, reorth)
            coeffs[(kind, x, x)] = (a, bsq)
            Gd.append(cf_green(a, bsq, z, E0, kind))
            G[:, x, x] += Gd[x]
        for x in range(p):
            for y in range(x + 1, p):
                a, bsq = lanczos_coefficients(opx.matvec, phis[x] + phis[y], max_steps, btol, reorth)
                coeffs[(kind, x, y)] = (a, bsq)
                gp = cf_green(a, bsq, z, E0, kind)
                gxy = 0.5 * (gp - Gd[x] - Gd[y])
                G[:, x, y] += gxy
                G[:, y, x] += gxy
    return G, coeffs


def band_lanczos_lehmann(matvec, Phi, max_dim, dtol=1e-10):
    """Lehmann pair (Q, lam) of H on the block Krylov subspace of Sec. 4.4.

    The subspace is span{phi_1..phi_p, H phi_1..H phi_p, H^2 phi_1, ...}.  Its orthonormal
    basis is built one vector at a time in that order (candidates queue; each accepted
    vector v_n enqueues H v_n), with full Gram-Schmidt (twice) and deflation of candidates
    whose remaining norm is below dtol times their norm before orthogonalization.  The
    projection T = V^T H V is diagonalized, T = S diag(lam) S^T, and Q = (V^T Phi)^T S
    (shape p x R): the projections of the phi_mu on the eigenvectors of T.
    """
    Phi = np.asarray(Phi, dtype=np.float64)
    queue = [Phi[:, k].copy() for k in range(Phi.shape[1])]
    V, HV = [], []
    while queue and len(V) < max_dim:
        c = queue.pop(0)
        n0 = np.linalg.norm(c)
        if n0 == 0.0:
            continue
        for _ in range(2):
            for v in V:
                c -= (v @ c) * v
        nc = np.linalg.norm(c)
        if nc < dtol * n0:
            continue
        v = c / nc
        V.append(v)
        w = matvec(v)
        HV.append(w)
        queue.append(w.copy())
    Vm = np.stack(V, axis=1)
    T = Vm.T @ np.stack(HV, axis=1)
    T = 0.5 * (T + T.T)
    lam, S = np.linalg.eigh(T)
    Q = (Vm.T @ Phi).T @ S
    return Q, lam


def green_band(model, n_up, n_dn, z, spin=0, orbitals=None, max_dim=600, dtol=1e-10, ground=None):
    """G_ij(z) from the band-Lanczos Lehmann representation (Sec. 4.4), electron and hole
    parts concatenated.  Returns (G[nz, p, p], Q[p, R], w[R])."""
    orbitals = list(range(model.ns)) if orbitals is None else list(orbitals)
    op = sector_hamiltonian(model, n_up, n_dn)
    if ground is None:
        E0, Om, _ = ground_state(op)
    else:
        E0, Om = ground
    Qs, ws = [], []
    for kind in ("e", "h"):
        nu = n_up + (1 if kind == "e" else -1) * (spin == 0)
        nd = n_dn + (1 if kind == "e" else -1) * (spin == 1)
        if nu < 0 or nd < 0 or nu > model.L or nd > model.L:
            continue
        opx = sector_hamiltonian(model, nu, nd)
        f = apply_cdag if kind == "e" else apply_c
        Phi = np.stack([f(model, n_up, n_dn, Om, i, spin).reshape(-1) for i in orbitals], axis=1)
        Q, lam = band_lanczos_lehmann(opx.matvec, Phi, max_dim, dtol)
        Qs.append(Q)
        ws.append(lam - E0 if kind == "e" else E0 - lam)
    Q = np.concatenate(Qs, axis=1)
    w = np.concatenate(ws)
    return lehmann_green(Q, w, z), Q, w


# ---------------------------------------------------------------------------------------
# Several low-lying states and mixed-state Green functions (Sec. 4.2, the library's
# Davidson_states and temperature options of Sec. 9)
# ---------------------------------------------------------------------------------------

def low_states(op, k, dense_limit=6000, tol=1e-13):
    """The k lowest eigenpairs of H in the sector: energies E[k] (ascending) and states
    V[k, d_up, d_dn] (unit norm).  Dense LAPACK up to dense_limit states, else ARPACK."""
    if op.dim <= dense_limit:
        w, V = np.linalg.eigh(op.sparse().toarray())
        w, V = w[:k], V[:, :k]
    else:
        v0 = np.cos(np.arange(op.dim) * 0.7) + 1.0
        w, V = spla.eigsh(op.linear_operator(), k=k, which="SA", tol=tol, v0=v0, ncv=max(24, 3 * k + 1))
        order = np.argsort(w)
        w, V = w[order], V[:, order]
    return w, np.stack([V[:, s].reshape(op.shape2) for s in range(len(w))])


def mixed_weights(E, T, degenerate_tol=1e-9):
    """Weights p_s of the low-lying states in the mixed state of temperature T: Boltzmann factors
    exp(-(E_s - E_0) / T) normalized over the states given; at T = 0 equal weights on the states
    within degenerate_tol max(1, |E_0|) of E_0 (the T -> 0 limit over a degenerate manifold)."""
    E = np.asarray(E, dtype=np.float64)
    if T > 0:
        w = np.exp(-(E - E[0]) / T)
    else:
        w = (E - E[0] <= degenerate_tol * max(1.0, abs(E[0]))).astype(np.float64)
    return w / w.sum()


def green_mixed(model, n_up, n_dn, z, k, T=0.0, spin=0, orbitals=None):
    """G(z) = sum_s p_s G_s(z) over the k lowest states s of the sector (mixed_weights), each G_s
    the exact Lehmann sum (Eq. spectral1) with E_s in place of E_0.  Returns (G, E, p)."""
    op = sector_hamiltonian(model, n_up, n_dn)
    E, V = low_states(op, k)
    p = mixed_weights(E, T)
    G = 0.0
    for s in range(len(E)):
        if p[s] == 0.0:
            continue
        G = G + p[s] * green_exact(model, n_up, n_dn, z, spin=spin, orbitals=orbitals, state=(E[s], V[s]))[0]
    return G, E, p
