"""FP64 CPU oracle of the lattice steps that consume the cluster Green function: cluster
perturbation theory (Sec. 3) and the CDMFT bath fit (Sec. 6).

TEST INFRASTRUCTURE ONLY (like ed_oracle): imported by ``tests/`` and ``bench.py``'s CPU legs,
never by the product package, and it imports nothing from it.

Conventions (those of ed_oracle): the one-body term is ``sum_ij t_ij c+_i c_j`` (a hopping "t = -1"
is the matrix element -1); the chemical potential enters the cluster block as ``h_c = t_c - mu``.
Frequencies ``z`` are complex arrays (``omega + i eta`` or ``i omega_n``); Green functions are
complex arrays ``G[nz, L, L]``.

The lattice is tiled by identical clusters of L sites (Sec. 2): site R of the cluster at
super-lattice vector r~ sits at r = r~ + R, r~ = n E for an integer vector n and the
super-lattice basis E (rows e_1 .. e_D).  A lattice model is given by the cluster's site
positions ``pos[L, D]``, the basis ``E[D, D]`` and a list of inter-cluster bonds ``(i, j, n, t)``:
the hopping matrix element ``t_{R_i, r~ + R_j} = t`` between site i of the cluster at the origin
and site j of the cluster at r~ = n E (its Hermitian partner, from that cluster back to site i, is
implied).  Hops inside the cluster are its own ``t_c`` matrix.

Parity status (pins in tests/test_lattice_oracle_pins.py):

* mixed_hopping: pinned (the worked L = 2 chain example of Sec. 2.2; Hermiticity).
* cpt_green, periodize: pinned (CPT is exact at U = 0 (Sec. 3.3): the periodized G equals
  1 / (z - eps(k)) of the lattice dispersion, chain and square lattice).
* hybridization: pinned (Schur complement of the full one-body resolvent: at U = 0 the cluster
  block of (z - h)^-1 equals (z - h_c - Gamma(z))^-1; one bath orbital in closed form).
* superlattice_average: pinned (at U = 0 it equals the cluster block of the real-space resolvent
  of the finite periodic lattice of N clusters).
* self_energy, cdmft_target, cdmft_distance: pinned (Sigma = 0 at U = 0; the distance vanishes
  at the bath parameters that generated its target and is positive elsewhere).
"""

from __future__ import annotations

import numpy as np


def mixed_hopping(t_c, bonds, E, kt):
    """t(k~)_{R R'} = sum_{r~} exp(i k~ . r~) t_{R, r~ + R'} (Sec. 2.2, mixed representation):
    the cluster's own hops t_c plus, for every inter-cluster bond (i, j, n, t) with r~ = n E,
    t e^{i k~.r~} at (i, j) and its Hermitian partner conj(t e^{i k~.r~}) at (j, i).
    kt: (D,) or (nk, D).  Returns complex (L, L) or (nk, L, L)."""
    t_c = np.asarray(t_c, dtype=np.float64)
    E = np.atleast_2d(np.asarray(E, dtype=np.float64))
    kt = np.asarray(kt, dtype=np.float64)
    single = kt.ndim == 1
    K = np.atleast_2d(kt)
    out = np.repeat(t_c[None].astype(np.complex128), len(K), axis=0)
    for i, j, n, t in bonds:
        rt = np.atleast_1d(np.asarray(n, dtype=np.float64)) @ E
        ph = t * np.exp(1j * (K @ rt))
        out[:, i, j] += ph
        out[:, j, i] += np.conj(ph)
    return out[0] if single else out


def inter_cluster(bonds, L, E, kt):
    """V(k~): the inter-cluster part of the mixed representation (Eq. CPT1)."""
    return mixed_hopping(np.zeros((L, L)), bonds, E, kt)


def hybridization(theta, eps, z):
    """Gamma_{mu nu}(z) = sum_a theta_{mu a} theta*_{nu a} / (z - eps_a) (Eq. hybridization).
    theta: (L, nb) real, eps: (nb,), z: (nz,).  Returns complex (nz, L, L)."""
    theta = np.asarray(theta, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    z = np.asarray(z, dtype=np.complex128).ravel()
    g = 1.0 / (z[:, None] - eps[None, :])                       # (nz, nb)
    return np.einsum("ma,na,ka->kmn", theta, theta, g)


def cpt_green(Gc, V, Gamma=None):
    """G(k~, z) = [G_c(z)^-1 (+ Gamma(z)) - V(k~)]^-1: Eq. CPT1, with the bath compensation of
    Eq. CPT_CDMFT when Gamma is given.  Gc: (nz, L, L); V: (nk, L, L).  Returns (nk, nz, L, L)."""
    Gci = np.linalg.inv(np.asarray(Gc, dtype=np.complex128))
    if Gamma is not None:
        Gci = Gci + Gamma
    M = Gci[None, :, :, :] - np.asarray(V)[:, None, :, :]
    return np.linalg.inv(M)


def periodize(G, pos, k):
    """G_per(k, z) = (1/L) sum_{R R'} exp(-i k . (R - R')) G_{R R'}(k, z) (Eq. CPT3, G scheme, with
    k~ replaced by k as the paper allows).  G: (nk, nz, L, L) computed at the same k; pos: (L, D);
    k: (nk, D).  Returns (nk, nz)."""
    pos = np.asarray(pos, dtype=np.float64)
    k = np.atleast_2d(np.asarray(k, dtype=np.float64))
    ph = np.exp(-1j * (k @ pos.T))                              # (nk, L): e^{-i k.R}
    L = pos.shape[0]
    return np.einsum("kr,kzrs,ks->kz", ph, G, np.conj(ph)) / L


def superlattice_average(Gc, V, Gamma=None):
    """G_bar(z) = (L/N) sum_{k~} [G_0^-1(k~) - Sigma_c(z)]^-1 (CDMFT step 3), written as the mean
    over the N/L reduced wave vectors of the CPT Green function of Eq. CPT_CDMFT (G_0^-1(k~) -
    Sigma_c = G_c^-1 + Gamma - V(k~)).  Returns (nz, L, L)."""
    return cpt_green(Gc, V, Gamma).mean(axis=0)


def self_energy(Gc, z, h_c, Gamma=None):
    """Sigma_c(z) = z - h_c - Gamma(z) - G_c(z)^-1 (Sec. 6: G_c^-1 = z - t_c - Gamma - Sigma_c)."""
    z = np.asarray(z, dtype=np.complex128).ravel()
    L = h_c.shape[0]
    S = z[:, None, None] * np.eye(L) - h_c[None] - np.linalg.inv(Gc)
    if Gamma is not None:
        S = S - Gamma
    return S


def cdmft_target(Gc, z, h_c, Gamma, V):
    """The fixed part of the CDMFT distance (Sec. 6, steps 3-4): Sigma_c from G_c and the current
    bath, G_bar from the super-lattice average, calG_0^-1 = G_bar^-1 + Sigma_c, and
    A(z) = z - h_c - calG_0^-1(z), so that d = sum_n W_n |A(z_n) - Gamma'(z_n)|^2 for a trial
    bath Gamma'.  Returns A (nz, L, L)."""
    z = np.asarray(z, dtype=np.complex128).ravel()
    L = h_c.shape[0]
    S = self_energy(Gc, z, h_c, Gamma)
    Gbar = superlattice_average(Gc, V, Gamma)
    G0i = np.linalg.inv(Gbar) + S
    return z[:, None, None] * np.eye(L) - h_c[None] - G0i


def cdmft_distance(theta, eps, z, W, A):
    """d = sum_n W_n sum_{nu nu'} |(z_n - h_c - Gamma(z_n) - calG_0^-1(z_n))_{nu nu'}|^2
    (Eq. dist_func) = sum_n W_n ||A(z_n) - Gamma(z_n)||_F^2 with A from cdmft_target."""
    R = np.asarray(A) - hybridization(theta, eps, z)
    return float(np.sum(np.asarray(W, dtype=np.float64)[:, None, None] * np.abs(R) ** 2))


def real_space_lattice(t_c, bonds, ncells):
    """One-body matrix of the finite periodic lattice of prod(ncells) clusters, cells indexed by
    integer vectors c (super-lattice vector c E): block (c, c) = t_c and, for every bond
    (i, j, n, t), t at (site i of cell c, site j of cell c + n) and its transpose, wrapped
    periodically.  Returns (N L, N L) real and the list of cell vectors."""
    t_c = np.asarray(t_c, dtype=np.float64)
    L = t_c.shape[0]
    ncells = [int(x) for x in ncells]
    cells = [np.array(c) for c in np.ndindex(*ncells)]
    index = {tuple(c): n for n, c in enumerate(cells)}
    N = len(cells)
    T = np.zeros((N * L, N * L))
    for n, c in enumerate(cells):
        T[n * L:(n + 1) * L, n * L:(n + 1) * L] += t_c
        for i, j, nv, t in bonds:
            m = index[tuple((c + np.atleast_1d(np.asarray(nv, dtype=int))) % ncells)]
            T[n * L + i, m * L + j] += t
            T[m * L + j, n * L + i] += t
    return T, cells
