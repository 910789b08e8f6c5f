"""Parity of the lattice kernels (CPT, Sec. 3; CDMFT bath fit, Sec. 6) with the lattice oracle.

The kernels take the cluster Green function as an input array, so the kernel parity tests feed
both sides the same oracle-computed G_c (host arrays from oracle/): FP64 complex inversions agree
to ~1e-13 relative; 1e-10 is asserted.  End-to-end tests run the CUDA solver's own G_c through
the kernels: at U = 0 CPT must give 1 / (z - eps(k)) exactly (Sec. 3.3), and one CDMFT iteration
must give the oracle's target and a fit that lowers the distance of Eq. dist_func.
"""

import numpy as np
import pytest

import oracle as O
import oracle_memo as OM
from oracle import lattice_oracle as LO
from paper_2305_18643_gb300 import build, ed
from paper_2305_18643_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def libed():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return ed.lib()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def _plaquette_impurity():
    """2x2 plaquette (t = -1, t' = 0.3) with 4 bath orbitals, U = 4, half filling of 8 orbitals."""
    rng = np.random.default_rng(31)
    T = W.lattice_hopping(2, 2, tp=0.3)
    eps = rng.uniform(-1.5, 1.5, 4)
    theta = np.zeros((4, 4))
    theta[np.arange(4), np.arange(4)] = rng.uniform(0.3, 0.7, 4)
    return W._cluster("plaquette+4 bath", T, 4.0, 2.0, 4, 4, eps, theta)


@pytest.fixture(scope="module")
def plaquette_gc():
    c = _plaquette_impurity()
    m = O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])
    om = W.matsubara_grid(96, 50.0)
    z = 1j * om
    Gc, Q, w, E0, gap = OM.green_exact(m, 4, 4, z)
    return c, m, om, z, Gc


def test_hybridization_matches_oracle():
    rng = np.random.default_rng(1)
    theta, eps = rng.uniform(-0.8, 0.8, (5, 7)), rng.uniform(-2, 2, 7)
    z = np.concatenate([1j * W.matsubara_grid(64, 50.0), W.real_grid(65) + 0.05j])
    G = ed.ed_hybridization(theta, eps, z)
    assert _rel(G, LO.hybridization(theta, eps, z)) <= 1e-13


@pytest.mark.parametrize("mode", [ed.ED_CPT_MATRIX, ed.ED_CPT_PERIODIZED, ed.ED_CPT_AVERAGE],
                         ids=["matrix", "periodized", "average"])
def test_cpt_kernels_match_oracle(plaquette_gc, mode):
    """The same oracle G_c (interacting plaquette with bath, Matsubara axis) on both sides; the
    square lattice tiled by 2x2 clusters; Gamma compensation of Eq. CPT_CDMFT included."""
    c, m, om, z, Gc = plaquette_gc
    lat = W.square_superlattice(2, 2, t=-1.0, tp=0.3)
    Gam = LO.hybridization(c["theta"], c["eps"], z)
    if mode == ed.ED_CPT_AVERAGE:
        kt = W.reduced_zone(lat["E"], (6, 6))
    else:
        kt = np.random.default_rng(2).uniform(-np.pi, np.pi, (23, 2))
    got = ed.ed_cpt_green(lat, Gc, kt, mode=mode, Gamma=Gam)
    V = LO.inter_cluster(lat["bonds"], 4, lat["E"], kt)
    if mode == ed.ED_CPT_AVERAGE:
        want = LO.superlattice_average(Gc, V, Gam)
    else:
        want = LO.cpt_green(Gc, V, Gam)
        if mode == ed.ED_CPT_PERIODIZED:
            want = LO.periodize(want, lat["pos"], kt)
    assert got.shape == want.shape
    assert _rel(got, want) <= 1e-10


@pytest.mark.parametrize("L", [1, 3, 16, 32])
def test_cpt_sizes_and_ragged_batches(L):
    """Chains tiled by L-site clusters (L = 1 .. 32 lanes of a warp) with a ragged number of
    (k, z) pairs; G_c = (z - t_c)^-1 so that the periodized result is 1 / (z - 2 t cos k)."""
    t = -0.8
    lat = W.square_superlattice(L, 1, t=t)
    z = np.array([0.3 + 0.2j, -1.0 + 0.05j, 2.2j, 0.1 + 1.0j, -2.5 + 0.3j])
    Gc = np.linalg.inv(z[:, None, None] * np.eye(L) - lat["t_c"][None])
    k = np.linspace(-np.pi, np.pi, 13)[:, None]
    Gp = ed.ed_cpt_green(lat, Gc, k, mode=ed.ED_CPT_PERIODIZED)
    want = 1.0 / (z[None, :] - 2 * t * np.cos(k))
    assert np.max(np.abs(Gp - want)) <= 1e-11


def test_cpt_exact_at_u0_through_the_solver():
    """End to end: the CUDA solver's G_c of a 2x2 plaquette at U = 0 (half filling, Matsubara
    axis) through the CPT kernels gives the square-lattice 1 / (z - eps(k)) (Sec. 3.3)."""
    t, tp = -1.0, 0.0
    lat = W.square_superlattice(2, 2, t=t, tp=tp)
    c = W._cluster("plaquette U=0", lat["t_c"], 0.0, 0.5, 2, 2)
    om = W.matsubara_grid(32, 50.0)
    with ed.Cluster(c) as cl:
        st, G = ed.ed_green(cl.h, om, 0.0, 4, axis=ed.ED_AXIS_MATSUBARA)
    k = np.random.default_rng(4).uniform(-np.pi, np.pi, (11, 2))
    Gp = ed.ed_cpt_green(lat, G, k, mode=ed.ED_CPT_PERIODIZED)
    eps = 2 * t * (np.cos(k[:, 0]) + np.cos(k[:, 1])) - c["mu"]
    want = 1.0 / (1j * om[None, :] - eps[:, None])
    assert np.max(np.abs(Gp - want)) <= 1e-8


def test_cdmft_target_matches_oracle(plaquette_gc):
    c, m, om, z, Gc = plaquette_gc
    lat = W.square_superlattice(2, 2, t=-1.0, tp=0.3)
    kt = W.reduced_zone(lat["E"], (8, 8))
    Gam = LO.hybridization(c["theta"], c["eps"], z)
    A = ed.ed_cdmft_target(lat, Gc, kt, Gamma=Gam)
    V = LO.inter_cluster(lat["bonds"], 4, lat["E"], kt)
    want = LO.cdmft_target(Gc, z, m.h[:4, :4], Gam, V)
    assert _rel(A, want) <= 1e-10


def test_distance_and_gradient_match_oracle(plaquette_gc):
    """Distances of several trial baths against the oracle's Eq. dist_func, and the analytic
    gradient against central differences of the oracle's distance."""
    c, m, om, z, Gc = plaquette_gc
    lat = W.square_superlattice(2, 2, t=-1.0, tp=0.3)
    kt = W.reduced_zone(lat["E"], (6, 6))
    Gam = LO.hybridization(c["theta"], c["eps"], z)
    A = LO.cdmft_target(Gc, z, m.h[:4, :4], Gam, LO.inter_cluster(lat["bonds"], 4, lat["E"], kt))
    Wn = 1.0 / om  # weights favouring low frequencies
    rng = np.random.default_rng(7)
    th = c["theta"][None] + 0.05 * rng.standard_normal((5, 4, 4))
    ep = c["eps"][None] + 0.1 * rng.standard_normal((5, 4))
    d, g = ed.ed_cdmft_distance(th, ep, z, Wn, A, grad=True)
    for q in range(5):
        assert abs(d[q] - LO.cdmft_distance(th[q], ep[q], z, Wn, A)) <= 1e-11 * max(1.0, d[q])
    h = 1e-6
    for p in [0, 3, 4 + 0 * 4 + 0, 4 + 2 * 4 + 2, 4 + 1 * 4 + 3]:
        e1, e2, t1, t2 = ep[0].copy(), ep[0].copy(), th[0].copy(), th[0].copy()
        if p < 4:
            e1[p] += h
            e2[p] -= h
        else:
            mu, a = divmod(p - 4, 4)
            t1[mu, a] += h
            t2[mu, a] -= h
        fd = (LO.cdmft_distance(t1, e1, z, Wn, A) - LO.cdmft_distance(t2, e2, z, Wn, A)) / (2 * h)
        assert abs(g[0, p] - fd) <= 1e-5 * max(1.0, abs(fd)), (p, g[0, p], fd)


def test_bath_fit_recovers_a_generating_bath():
    """Step 4 of the CDMFT loop on a target that a known bath produces exactly: from a perturbed
    start the fit drives the distance to ~0 and reproduces that bath's hybridization function
    (parameters themselves are unique only up to symmetries, Gamma is not)."""
    rng = np.random.default_rng(11)
    L, nb = 2, 4
    th0 = np.zeros((L, nb))
    th0[np.arange(nb) % L, np.arange(nb)] = rng.uniform(0.3, 0.8, nb)
    ep0 = np.array([-1.2, -0.4, 0.5, 1.3])
    om = W.matsubara_grid(128, 50.0)
    z = 1j * om
    A = LO.hybridization(th0, ep0, z)  # A = Gamma* exactly: d vanishes at (th0, ep0)
    free = th0 != 0.0
    th, ep, d, it = ed.ed_cdmft_fit(th0 * 1.3, ep0 + 0.2, z, np.ones(len(om)), A, theta_free=free)
    assert d <= 1e-16, (d, it)
    assert np.all(th[~free] == 0.0)
    assert np.max(np.abs(LO.hybridization(th, ep, z) - A)) <= 1e-7


def test_cdmft_iteration_through_the_solver():
    """One CDMFT iteration on the 1D Hubbard chain tiled by 2-site clusters with 4 bath orbitals
    (U = 4, half filling; cf. the 1D example of Sec. 6): G_c from the CUDA solver on the
    Matsubara axis, the target from the lattice kernels, then the bath fit.  The target agrees
    with the oracle's (computed from the oracle's own G_c), and the fit lowers the distance."""
    lat = W.square_superlattice(2, 1, t=-1.0)
    theta = np.array([[0.5, 0.0, 0.4, 0.0], [0.0, 0.5, 0.0, 0.4]])
    eps = np.array([-1.0, -1.0, 1.0, 1.0])
    c = W._cluster("chain2+4 bath", lat["t_c"], 4.0, 2.0, 3, 3, eps, theta)
    m = O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])
    om = W.matsubara_grid(128, 50.0)
    z = 1j * om
    kt = W.reduced_zone(lat["E"], (64,))
    with ed.Cluster(c) as cl:
        st, Gc = ed.ed_green(cl.h, om, 0.0, 2, axis=ed.ED_AXIS_MATSUBARA)
    Gam = ed.ed_hybridization(theta, eps, z)
    A = ed.ed_cdmft_target(lat, Gc, kt, Gamma=Gam)
    Gc_o = OM.green_exact(m, 3, 3, z)[0]
    A_o = LO.cdmft_target(Gc_o, z, m.h[:2, :2], LO.hybridization(theta, eps, z),
                          LO.inter_cluster(lat["bonds"], 2, lat["E"], kt))
    assert np.max(np.abs(A - A_o)) <= 1e-7 * max(1.0, np.max(np.abs(A_o)))
    Wn = np.ones(len(om))
    d0 = LO.cdmft_distance(theta, eps, z, Wn, A_o)
    th, ep, d, it = ed.ed_cdmft_fit(theta, eps, z, Wn, A, theta_free=theta != 0.0)
    assert d < d0
    assert abs(LO.cdmft_distance(th, ep, z, Wn, A_o) - d) <= 1e-6 * max(1.0, d)
