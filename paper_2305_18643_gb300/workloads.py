"""Seeded synthetic cluster generators (inputs only; none of the solver's arithmetic).

Both the CUDA path's tests/bench and the CPU oracle receive clusters from here as plain
arrays.  A cluster is a dict::

    {"name": str, "t": (ns, ns) float64 symmetric, "U": (ns,) float64, "mu": float,
     "eps": (nb,) float64, "theta": (ns, nb) float64, "n_up": int, "n_dn": int}

Sites of a W x H lattice are numbered s = x + W * y.  Hopping amplitudes are matrix
elements t_ij of the one-body term sum t_ij c+_i c_j (nearest neighbour t = -1).
Seeds: 20230529 + 1000 * workload_index + instance.
"""

from __future__ import annotations

import numpy as np

SEED_BASE = 20230529


def seed_for(workload_index, instance=0):
    return SEED_BASE + 1000 * workload_index + instance


def _cluster(name, t, U, mu, n_up, n_dn, eps=None, theta=None):
    ns = t.shape[0]
    eps = np.zeros(0) if eps is None else np.asarray(eps, dtype=np.float64)
    theta = np.zeros((ns, len(eps))) if theta is None else np.asarray(theta, dtype=np.float64)
    return {"name": name, "t": np.ascontiguousarray(t, dtype=np.float64),
            "U": np.broadcast_to(np.asarray(U, dtype=np.float64), (ns,)).copy(), "mu": float(mu),
            "eps": eps, "theta": theta.reshape(ns, len(eps)), "n_up": int(n_up), "n_dn": int(n_dn)}


def lattice_hopping(W, H, t=-1.0, tp=0.0, periodic=False, rng=None, seeded_tp_sign=False):
    """Nearest-neighbour (t) and diagonal (tp) hopping on a W x H lattice, s = x + W y.

    With ``periodic`` both directions wrap (bonds are added once; on a length-2 direction
    the wrap bond coincides with the direct one and is skipped).  With ``seeded_tp_sign``
    every diagonal bond gets tp * s_b, s_b = +-1 drawn from ``rng``.
    """
    n = W * H
    T = np.zeros((n, n))
    bonds = set()

    def add(i, j, v):
        if i == j:
            return
        key = (min(i, j), max(i, j))
        if key in bonds:
            return
        bonds.add(key)
        T[i, j] = T[j, i] = v

    for y in range(H):
        for x in range(W):
            s = x + W * y
            for dx, dy in ((1, 0), (0, 1)):
                xx, yy = x + dx, y + dy
                if periodic:
                    xx, yy = xx % W, yy % H
                elif xx >= W or yy >= H:
                    continue
                add(s, xx + W * yy, t)
    if tp != 0.0:
        for y in range(H):
            for x in range(W):
                s = x + W * y
                for dx, dy in ((1, 1), (-1, 1)):
                    xx, yy = x + dx, y + dy
                    if periodic:
                        xx, yy = xx % W, yy % H
                    elif not (0 <= xx < W and 0 <= yy < H):
                        continue
                    v = tp
                    if seeded_tp_sign:
                        v = tp * (1.0 if rng.random() < 0.5 else -1.0)
                    add(s, xx + W * yy, v)
    return T


def plain_2x4(U=4.0):
    """8-site 2x4 open Hubbard cluster, t = -1, U = 4, mu = U/2, N_up = N_dn = 4 (d = 4,900)."""
    T = lattice_hopping(4, 2)
    return _cluster("2x4 open, U=4, half filling", T, U, U / 2, 4, 4)


def open_3x4_c2v(U=4.0):
    """12-site 3x4 open Hubbard cluster (W = 4, H = 3, s = x + 4 y), t = -1, U = 4, mu = U/2,
    N_up = N_dn = 6 (d = 853,776): the cluster of Table 1 with an interaction.  Also returns its
    two mirror generators m_x: x -> 3 - x and m_y: y -> 2 - y (orbital images), whose group C2v
    leaves H invariant."""
    T = lattice_hopping(4, 3)
    mx = [(3 - s % 4) + 4 * (s // 4) for s in range(12)]
    my = [s % 4 + 4 * (2 - s // 4) for s in range(12)]
    return _cluster("3x4 open, U=4, half filling", T, U, U / 2, 6, 6), [mx, my]


def cdmft_2x2_bath(instance=0):
    """2x2 plaquette (t = -1, t' = +0.3, U = 8, mu = 4) plus 8 bath orbitals, N_up = N_dn = 6.

    Bath orbital a (0..7) couples to site a mod 4 with theta ~ U[0.2, 0.8]; eps ~ U[-2, 2].
    Sector dimension 924^2 = 853,776.
    """
    rng = np.random.default_rng(seed_for(1, instance))
    T = lattice_hopping(2, 2, tp=0.3)
    eps = rng.uniform(-2.0, 2.0, 8)
    theta = np.zeros((4, 8))
    theta[np.arange(8) % 4, np.arange(8)] = rng.uniform(0.2, 0.8, 8)
    return _cluster("2x2 plaquette + 8 bath, U=8", T, 8.0, 4.0, 6, 6, eps, theta)


def periodic_4x4(instance=0):
    """16-site 4x4 periodic cluster, t = -1, t' = 0.3 s_b (seeded sign per diagonal bond),
    U = 8, mu = 4, N_up = N_dn = 8 (d = 12,870^2 = 165,636,900)."""
    rng = np.random.default_rng(seed_for(2, instance))
    T = lattice_hopping(4, 4, tp=0.3, periodic=True, rng=rng, seeded_tp_sign=True)
    return _cluster("4x4 periodic, U=8, half filling", T, 8.0, 4.0, 8, 8)


def batched_family(n_clusters=512, instance=0, min_orb=4, max_orb=12):
    """Seeded family of small clusters: open chains, 2-leg ladders and 2x2 plaquettes with
    0..8 bath orbitals; 4..12 orbitals in total; |t| ~ U[0.5, 1.5] per bond; U ~ U[2, 10];
    mu = U/2; random fillings N_up, N_dn in [1, n - 1]."""
    rng = np.random.default_rng(seed_for(3, instance))
    out = []
    while len(out) < n_clusters:
        kind = int(rng.integers(0, 3))
        if kind == 0:
            ns, nb = int(rng.integers(min_orb, max_orb + 1)), 0
            T = lattice_hopping(ns, 1)
        elif kind == 1:
            W = int(rng.integers(2, max_orb // 2 + 1))
            ns, nb = 2 * W, 0
            T = lattice_hopping(W, 2)
        else:
            ns = 4
            nb = int(rng.integers(max(0, min_orb - 4), min(8, max_orb - 4) + 1))
            T = lattice_hopping(2, 2)
        if not (min_orb <= ns + nb <= max_orb):
            continue
        mag = rng.uniform(0.5, 1.5, size=T.shape)
        mag = np.triu(mag, 1)
        mag = mag + mag.T
        T = T * mag
        U = float(rng.uniform(2.0, 10.0))
        eps = rng.uniform(-2.0, 2.0, nb)
        theta = np.zeros((ns, nb))
        if nb:
            theta[np.arange(nb) % ns, np.arange(nb)] = rng.uniform(0.2, 0.8, nb)
        n = ns + nb
        n_up = int(rng.integers(1, n))
        n_dn = int(rng.integers(1, n))
        out.append(_cluster(f"batched#{len(out)} ({'chain ladder plaquette'.split()[kind]}, n={n})",
                            T, U, U / 2, n_up, n_dn, eps, theta))
    return out


def served_request(rng, sizes=(8, 10, 12, 14)):
    """One served solve request: a 2 x W open cluster (W = n/2) with t = -1, t' = +-0.3 seeded
    per diagonal bond, U = 8, mu = 4, half filling."""
    n = int(sizes[int(rng.integers(0, len(sizes)))])
    T = lattice_hopping(n // 2, 2, tp=0.3, rng=rng, seeded_tp_sign=True)
    return _cluster(f"served 2x{n // 2}", T, 8.0, 4.0, n // 2, n // 2)


def hubbard_dimer(t=-1.0, U=4.0, mu=0.0):
    """Two-site Hubbard cluster at half filling (N_up = N_dn = 1)."""
    T = np.array([[0.0, t], [t, 0.0]])
    return _cluster("dimer", T, U, mu, 1, 1)


def random_cluster(rng, ns, nb, n_up, n_dn, U=None, dense_t=False):
    """Random small cluster for parity tests: random symmetric t (dense or chain), random U,
    mu, bath energies and hybridizations."""
    if dense_t:
        T = rng.uniform(-1.0, 1.0, (ns, ns))
        T = 0.5 * (T + T.T)
    else:
        T = lattice_hopping(ns, 1) * rng.uniform(0.5, 1.5)
        T[np.diag_indices(ns)] = rng.uniform(-0.5, 0.5, ns)
    Uv = rng.uniform(1.0, 6.0, ns) if U is None else np.full(ns, float(U))
    eps = rng.uniform(-2.0, 2.0, nb)
    theta = rng.uniform(0.2, 0.8, (ns, nb))
    return _cluster("random", T, Uv, float(rng.uniform(0.0, 3.0)), n_up, n_dn, eps, theta)


def real_grid(n_freq=1000, lo=-8.0, hi=8.0):
    """Real-frequency grid with both end points: lo + (hi - lo) k / (n - 1)."""
    return lo + (hi - lo) * np.arange(n_freq) / (n_freq - 1)


def matsubara_grid(n_freq=2048, beta=50.0):
    """Fermionic Matsubara frequencies (2n + 1) pi / beta, n = 0 .. n_freq - 1."""
    return (2 * np.arange(n_freq) + 1) * np.pi / beta


def square_superlattice(W, H, t=-1.0, tp=0.0):
    """A square lattice (nearest-neighbour t, diagonal tp) tiled by W x H clusters (Sec. 2):
    returns {"t_c": (L, L) cluster hops, "pos": (L, 2) site positions (x, y) with s = x + W y,
    "E": super-lattice basis [[W, 0], [0, H]], "bonds": [(i, j, (n1, n2), t)]}.  A bond joins
    site i of the cluster at the origin to site j of the cluster at n1 e_1 + n2 e_2; every lattice
    bond leaving the cluster appears once (displacements (1,0), (0,1), (1,1), (-1,1) from each
    site).  H = 1 with tp = 0 is a chain tiled by W-site clusters."""
    L = W * H
    t_c = np.zeros((L, L))
    bonds = []
    pos = np.array([[s % W, s // W] for s in range(L)], dtype=np.float64)
    disps = [((1, 0), t), ((0, 1), t)] + ([((1, 1), tp), ((-1, 1), tp)] if tp != 0.0 else [])
    if H == 1:
        disps = [d for d in disps if d[0][1] == 0]
    for s in range(L):
        x, y = s % W, s // W
        for (dx, dy), v in disps:
            X, Y = x + dx, y + dy
            n1, n2 = X // W, Y // H
            j = (X - n1 * W) + W * (Y - n2 * H)
            if (n1, n2) == (0, 0):
                t_c[s, j] += v
                t_c[j, s] += v
            else:
                bonds.append((s, j, (n1, n2) if H > 1 else (n1,), v))
    E = np.array([[W, 0.0], [0.0, H]]) if H > 1 else np.array([[float(W)]])
    return {"t_c": t_c, "pos": pos if H > 1 else pos[:, :1], "E": E, "bonds": bonds}


def reduced_zone(E, ncells):
    """The prod(ncells) wave vectors k~ of the super-lattice Brillouin zone that a periodic
    lattice of ncells[a] clusters along e_a supports: k~ . e_a = 2 pi m_a / ncells[a]."""
    E = np.atleast_2d(np.asarray(E, dtype=np.float64))
    B = 2 * np.pi * np.linalg.inv(E).T          # rows b_a with b_a . e_b = 2 pi delta_ab
    ms = np.array(list(np.ndindex(*[int(n) for n in ncells])), dtype=np.float64)
    return (ms / np.asarray(ncells, dtype=np.float64)) @ B
