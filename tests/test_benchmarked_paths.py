"""Oracle parity of the code paths that the benchmark times, at sizes the oracle can check.

* Two-pass H.psi (a row pass for the down-spin hops and the diagonal, a column pass for the
  up-spin hops and the fused Lanczos reductions).  The library takes it for vectors of 32 MiB
  and more (the 4x4 workload, the 12/14-orbital band requests of the served form);
  ED_OPT_TWO_PASS_MIN_BYTES = 0 makes it run on small sectors, where ground energies and
  Green functions are checked against the oracle: E0 to 1e-10 relative (Sec. 4.2), G to 1e-8
  absolute (Eq. green, Sec. 4.3; band Lanczos of Sec. 4.4).  A 2x7 cluster (14 orbitals) takes
  it without the option.
* The FP32-storage form: ground energies to 1e-10 after the FP64 refinement, the FP64
  residual to 1e-12, and G within stated bounds of the oracle.
* The batched form's block-level continued fractions (runs of more than 8,192 states) at the
  library's default level cap, the cap the batched benchmark uses.
"""

import math
import os

import numpy as np
import pytest

import oracle as O
import oracle_memo as OM
from paper_2305_18643_gb300 import build, ed
from paper_2305_18643_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# FP32-storage G against the oracle (absolute, max over the grid and i, j).  FP32 vectors carry
# a relative rounding of 6e-8 per element; the starting vectors c+W alone move G by about
# 2 x 6e-8 x |G| (|G| <= 1/eta = 20 on the real axis at eta = 0.05, <= beta/pi = 16 at the lowest
# Matsubara frequency for beta = 50), and every level of the recursion adds rounding of the same
# size to coefficients whose errors the real axis amplifies near poles by up to 1/eta^2.  Measured
# on GB300 (the cases below and the batched clusters): up to 1.0e-4 on the real axis, below 5e-6
# on the Matsubara axis.  The bounds leave a factor 2 over the real-axis measurements.
FP32_G_TOL_REAL = 2e-4
FP32_G_TOL_MATSUBARA = 5e-6


@pytest.fixture(scope="module", autouse=True)
def libed():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return ed.lib()


def _model(c):
    return O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _force_two_pass(cl):
    ed.ed_set_option(cl.h, ed.ED_OPT_TWO_PASS_MIN_BYTES, 0)


def _three_magnitude_chain():
    """A 6-site ring with bond values -1, -0.5, +0.7: three magnitudes, so the row pass selects
    among the signed values (the 2x4 cluster and the 3x3 lattice below use the two-magnitude
    form, the random clusters the table of values in shared memory)."""
    T = np.zeros((6, 6))
    for i, v in enumerate([-1.0, -0.5, 0.7, -1.0, -0.5, 0.7]):
        j = (i + 1) % 6
        T[i, j] = T[j, i] = v
    return W._cluster("6-ring, three magnitudes", T, 4.0, 2.0, 3, 2)


SMALL = [("2x4", W.plain_2x4()),
         ("rand-bath", W.random_cluster(np.random.default_rng(3), 3, 3, 2, 4)),
         ("chain5", W.random_cluster(np.random.default_rng(4), 5, 0, 1, 4)),
         ("2x2+bath", W.cdmft_2x2_bath()),
         # t = -1 and t' = +-0.3 with seeded signs: two magnitudes, values of both signs
         ("3x3-tp-signs", W._cluster("3x3 open, t' of seeded sign", W.lattice_hopping(
             3, 3, tp=0.3, rng=np.random.default_rng(7), seeded_tp_sign=True), 8.0, 4.0, 5, 4)),
         ("ring6-3mag", _three_magnitude_chain())]


# ------------------------------------------------------------------ H.psi, element by element
@pytest.mark.parametrize("name,c", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("shift", [(0, 0), (1, 0), (0, -1)])
def test_two_pass_hpsi_matches_oracle(name, c, shift):
    """Rows padded to a multiple of 128 elements (the solver's own layout) and the option at 0:
    ed_hpsi runs the two-pass kernels.  d_up values of 70, 35, 10 and 924 leave ragged 4-row
    groups and 64-row blocks (also 126 and 20 for the last two clusters); every padding element
    must stay zero.  The clusters cover the three ways the row pass finds a hop's value."""
    m = _model(c)
    nu, nd = c["n_up"] + shift[0], c["n_dn"] + shift[1]
    if not (0 <= nu <= m.L and 0 <= nd <= m.L):
        pytest.skip("sector does not exist")
    op = O.sector_hamiltonian(m, nu, nd)
    du, dd = op.shape2
    ld = (dd + 127) // 128 * 128
    psi = np.random.default_rng(11).standard_normal((du, dd))
    with ed.Cluster(c) as cl:
        _force_two_pass(cl)
        for dtype, tdt, tol in ((ed.ED_FP64, torch.float64, 1e-12), (ed.ED_FP32, torch.float32, 2e-5)):
            x = torch.zeros((du, ld), dtype=tdt, device="cuda")
            x[:, :dd] = torch.as_tensor(psi, device="cuda").to(tdt)
            y = torch.zeros_like(x)
            ed.ed_hpsi(cl.h, nu, nd, dtype, x.data_ptr(), y.data_ptr(), ld, _stream())
            torch.cuda.synchronize()
            assert float(y[:, dd:].abs().max()) == 0.0, "padding written"
            ref = O.apply_h(op, x[:, :dd].double().cpu().numpy())
            got = y[:, :dd].double().cpu().numpy()
            assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_two_pass_option_changes_the_kernels():
    """With the option at 0 every fused Lanczos step is two launches (row pass, column pass)
    instead of one: the ground state of the 2x4 cluster launches at least one more kernel per
    Lanczos level, and reaches the same energy."""
    c = W.plain_2x4()
    counts, energies = [], []
    for force in (False, True):
        with ed.Cluster(c) as cl:
            if force:
                _force_two_pass(cl)
            n0 = ed.ed_launch_count()
            st, E, res, it = cl.ground_state()
            counts.append((ed.ed_launch_count() - n0, it))
            energies.append(E)
    (n_one, it_one), (n_two, it_two) = counts
    assert it_one == it_two
    assert n_two - n_one >= it_two
    assert abs(energies[0] - energies[1]) <= 1e-12 * abs(energies[0])


# ------------------------------------------------------------------ ground state and G, forced two-pass
@pytest.mark.parametrize("precision", [ed.ED_FP64, ed.ED_FP32], ids=["fp64", "fp32"])
def test_two_pass_ground_state_2x4(precision):
    c = W.plain_2x4()
    E0, Om, gap = OM.ground_state(_model(c), 4, 4)
    with ed.Cluster(c, precision=precision) as cl:
        _force_two_pass(cl)
        st, E, res, it = cl.ground_state()
        Wv = cl.ground_vector()
    assert st == ed.ED_OK
    assert abs(E - E0) <= 1e-10 * abs(E0)
    assert res <= 1e-12
    assert abs(abs(np.vdot(Wv, Om)) - 1.0) < 1e-10


@pytest.mark.parametrize("method", [ed.ED_GF_CF, ed.ED_GF_BAND], ids=["cf", "band"])
def test_two_pass_green_2x4(method):
    """2x4 open, U = 4, half filling: all 8 x 8 G_ij on 1000 real frequencies, eta = 0.05,
    against the exact Lehmann sum (Eq. spectral1), with the two-pass kernels in every run."""
    c = W.plain_2x4()
    om = W.real_grid(1000)
    Gref = OM.green_exact(_model(c), 4, 4, om + 0.05j)[0]
    with ed.Cluster(c, gf_method=method) as cl:
        _force_two_pass(cl)
        st, G = ed.ed_green(cl.h, om, 0.05, 8)
    assert st in (ed.ED_OK, ed.ED_WARN_DEGENERATE)
    assert np.max(np.abs(G - Gref)) <= 1e-8


GF_CASES = [("bath-asym", W.random_cluster(np.random.default_rng(21), 3, 3, 2, 4), 0),
            ("bath-down", W.random_cluster(np.random.default_rng(22), 3, 2, 3, 2), 1),
            ("nearly-full", W.random_cluster(np.random.default_rng(24), 4, 1, 5, 3), 0)]


@pytest.mark.parametrize("name,c,spin", GF_CASES, ids=[g[0] for g in GF_CASES])
@pytest.mark.parametrize("method", [ed.ED_GF_CF, ed.ED_GF_BAND], ids=["cf", "band"])
@pytest.mark.parametrize("axis", [ed.ED_AXIS_REAL, ed.ED_AXIS_MATSUBARA], ids=["real", "matsubara"])
def test_two_pass_green_matches_exact(name, c, spin, method, axis):
    m = _model(c)
    if axis == ed.ED_AXIS_REAL:
        om = W.real_grid(301)
        z = om + 0.05j
    else:
        om = W.matsubara_grid(256, 50.0)
        z = 1j * om
    Gref = OM.green_exact(m, c["n_up"], c["n_dn"], z, spin=spin)[0]
    with ed.Cluster(c, gf_method=method) as cl:
        _force_two_pass(cl)
        st, G = ed.ed_green(cl.h, om, 0.05, m.ns, axis=axis, spin=spin)
    assert np.max(np.abs(G - Gref)) <= 1e-8


@pytest.fixture(scope="module")
def cdmft_reference():
    """Oracle ground state of the 12-orbital impurity (2x2 plaquette + 8 bath, d = 853,776) and
    its band-Lanczos G on 6 blocks (24 Krylov vectors per part) on the Matsubara axis."""
    c = W.cdmft_2x2_bath()
    m = _model(c)
    op = O.sector_hamiltonian(m, 6, 6)
    E0, Om, gap = O.ground_state(op)
    om = W.matsubara_grid(128, 50.0)
    R = 24
    Gb = O.green_band(m, 6, 6, 1j * om, max_dim=R, ground=(E0, Om))[0]
    return c, E0, gap, om, R, Gb


@pytest.mark.parametrize("precision", [ed.ED_FP64, ed.ED_FP32], ids=["fp64", "fp32"])
def test_two_pass_cdmft_impurity(cdmft_reference, precision):
    """12 orbitals through the two-pass kernels: E0 to 1e-10, residual to 1e-12, and band G at
    24 Krylov vectors per part equal to the oracle's band Lanczos on the same block Krylov space
    (to 1e-8 with FP64 vectors; within the FP32 bound with FP32 vectors)."""
    c, E0, gap, om, R, Gb = cdmft_reference
    with ed.Cluster(c, precision=precision, gf_method=ed.ED_GF_BAND) as cl:
        _force_two_pass(cl)
        st, E, res, it = cl.ground_state()
        ed.ed_set_option(cl.h, ed.ED_OPT_BAND_MAX_DIM, R)
        ed.ed_set_option(cl.h, ed.ED_OPT_GF_TOL, 1e-300)
        stg, G = ed.ed_green(cl.h, om, 0.0, 4, axis=ed.ED_AXIS_MATSUBARA)
        tot, mx = ed.ed_green_stats(cl.h)
    assert st in (ed.ED_OK, ed.ED_WARN_DEGENERATE)
    assert abs(E - E0) <= 1e-10 * abs(E0)
    assert res <= 1e-12
    assert mx == R
    tol = 1e-8 if precision == ed.ED_FP64 else FP32_G_TOL_MATSUBARA
    assert np.max(np.abs(G - Gb)) <= tol


@pytest.fixture(scope="module")
def ladder14_reference():
    """2x7 open ladder, t = -1, t' = +-0.3, U = 8, mu = 4, half filling (d = 3432^2 =
    11,778,624; 94 MB per FP64 vector, so the library takes the two-pass kernels by itself).
    The oracle's E0 and band-Lanczos G on two blocks (28 Krylov vectors per part, 64 Matsubara
    frequencies) are stored in tests/golden/ladder14_band.npz by tests/golden/make_ladder14.py
    (ARPACK on 1.2e7 states takes minutes of CPU).  Two blocks of the 14 sites' starting vectors:
    28 Krylov vectors per part, the library's minimum run."""
    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ladder14_band.npz"))
    c = W.served_request(np.random.default_rng(int(g["seed"])), sizes=(14,))
    return c, float(g["E0"]), float(g["gap"]), g["omega"], int(g["R"]), g["G"]


@pytest.mark.parametrize("precision", [ed.ED_FP64, ed.ED_FP32], ids=["fp64", "fp32"])
def test_ladder14_natural_two_pass(ladder14_reference, precision):
    c, E0, gap, om, R, Gb = ladder14_reference
    with ed.Cluster(c, precision=precision, gf_method=ed.ED_GF_BAND) as cl:
        st, E, res, it = cl.ground_state()
        ed.ed_set_option(cl.h, ed.ED_OPT_BAND_MAX_DIM, R)
        ed.ed_set_option(cl.h, ed.ED_OPT_GF_TOL, 1e-300)
        stg, G = ed.ed_green(cl.h, om, 0.0, 14, axis=ed.ED_AXIS_MATSUBARA)
        tot, mx = ed.ed_green_stats(cl.h)
    assert st in (ed.ED_OK, ed.ED_WARN_DEGENERATE)
    assert abs(E - E0) <= 1e-10 * abs(E0)
    assert res <= 1e-12
    assert mx == R
    tol = 1e-8 if precision == ed.ED_FP64 else FP32_G_TOL_MATSUBARA
    assert np.max(np.abs(G - Gb)) <= tol


# ------------------------------------------------------------------ FP32-storage G against the oracle
FP32_CASES = [("2x4", W.plain_2x4(), 0), ("bath-asym", GF_CASES[0][1], 0), ("bath-down", GF_CASES[1][1], 1)]


@pytest.mark.parametrize("name,c,spin", FP32_CASES, ids=[g[0] for g in FP32_CASES])
@pytest.mark.parametrize("method", [ed.ED_GF_CF, ed.ED_GF_BAND], ids=["cf", "band"])
@pytest.mark.parametrize("axis", [ed.ED_AXIS_REAL, ed.ED_AXIS_MATSUBARA], ids=["real", "matsubara"])
def test_fp32_green_within_stated_bound(name, c, spin, method, axis):
    """FP32 vectors with FP64 recurrence: G against the exact Lehmann sum within the bounds
    stated at the top of this file; E0 to 1e-10 and the FP64 residual to 1e-12."""
    m = _model(c)
    if axis == ed.ED_AXIS_REAL:
        om = W.real_grid(301)
        z, tol = om + 0.05j, FP32_G_TOL_REAL
    else:
        om = W.matsubara_grid(256, 50.0)
        z, tol = 1j * om, FP32_G_TOL_MATSUBARA
    Gref, Q, w, E0, gap = OM.green_exact(m, c["n_up"], c["n_dn"], z, spin=spin)
    with ed.Cluster(c, precision=ed.ED_FP32, gf_method=method) as cl:
        st, E, res, it = cl.ground_state()
        stg, G = ed.ed_green(cl.h, om, 0.05, m.ns, axis=axis, spin=spin)
    assert abs(E - E0) <= 1e-10 * max(1.0, abs(E0))
    assert res <= 1e-12
    assert np.max(np.abs(G - Gref)) <= tol


# ------------------------------------------------------------------ batched form, block-level runs
def _big_runs_family():
    """Two clusters of the batched family with 9-10 orbitals whose hole sectors hold 8,192 -
    20,000 states (so their continued fractions run on whole thread blocks), at most 4 cluster
    sites (few continued fractions for the oracle) and n_up = n_dn (one spin)."""
    fam = W.batched_family(4000, instance=5, min_orb=9, max_orb=10)
    out = []
    for c in fam:
        L = len(c["eps"]) + c["t"].shape[0]
        if c["t"].shape[0] > 4 or c["n_up"] != c["n_dn"]:
            continue
        dm = math.comb(L, c["n_up"] - 1) * math.comb(L, c["n_dn"])
        if dm <= 8192 or dm > 20000:
            continue
        out.append(c)
        if len(out) == 2:
            break
    return out


@pytest.mark.parametrize("precision", [ed.ED_FP64, ed.ED_FP32], ids=["fp64", "fp32"])
def test_batch_block_level_runs_match_oracle(precision):
    """Batched solve at the library's default level cap (the cap of the batched benchmark):
    E0 to 1e-10 and, with FP64 vectors, G of the block-level continued fractions to 1e-8 of the
    oracle's continued fractions (Eq. jacobi, run to convergence); FP32 within its bound."""
    fam = _big_runs_family()
    assert len(fam) == 2
    om = W.real_grid(201)
    z = om + 0.05j
    E0, res, st, it, G = ed.ed_batch_solve(fam, precision=precision, omega=om, eta=0.05)
    for k, c in enumerate(fam):
        m = _model(c)
        op = O.sector_hamiltonian(m, c["n_up"], c["n_dn"])
        Eref, Om, gap = O.ground_state(op)
        assert abs(E0[k] - Eref) <= 1e-10 * max(1.0, abs(Eref)), (k, c["name"])
        if gap < 1e-6:
            continue  # degenerate ground state: G is not unique (Sec. 4.2)
        # both clusters reach an invariant subspace (b_n < 1e-10 b_0) before 3,000 levels
        Gref = O.green_cf(m, c["n_up"], c["n_dn"], z, spin=0, max_steps=3000, reorth=False,
                          ground=(Eref, Om))[0]
        tol = 1e-8 if precision == ed.ED_FP64 else FP32_G_TOL_REAL
        assert np.max(np.abs(G[k][0] - Gref)) <= tol, (k, c["name"], np.max(np.abs(G[k][0] - Gref)))
