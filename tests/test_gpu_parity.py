"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Integer work (basis, hopping tables) must be bit-exact.  Floating point: FP64 ground energies
within 1e-10 relative, FP64 G(omega) within 1e-8 absolute, FP64 H.psi within 1e-12 of max|y|
(rounding order only), FP32 H.psi within 2e-5 of max|y| (FP32 products and sums of <= 70 terms).
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_2305_18643_gb300 import build, ed
from paper_2305_18643_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def libed():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return ed.lib()


def _model(c):
    return O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])


def _stream():
    return torch.cuda.current_stream().cuda_stream


# ------------------------------------------------------------------ K1: basis (bit-exact)
@pytest.mark.parametrize("L", [1, 2, 5, 8, 12, 16, 20])
def test_basis_bit_exact(L):
    for N in sorted({0, 1, L // 2, L - 1, L}):
        if N < 0 or N > L:
            continue
        gpu = ed.ed_basis(L, N)
        ref = O.sector_basis(L, N)
        assert gpu.dtype == np.uint32 and len(gpu) == math.comb(L, N)
        assert np.array_equal(gpu.astype(np.uint64), ref)


# ------------------------------------------------------------------ K2: hopping tables (bit-exact)
def _gpu_table_tuples(h, N, L):
    ptr, ent, vals = ed.ed_hop_table(h, N, L)
    rows = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    cols = (ent >> 8).astype(np.int64)
    neg = ((ent >> 7) & 1).astype(np.int64)
    v = vals[(ent & 127).astype(np.int64)]
    return sorted(zip(rows.tolist(), cols.tolist(), neg.tolist(), v.tolist()))


def _oracle_table_tuples(hmat, N):
    row, col, a, b, sign = O.hop_entries(hmat, N)
    return sorted(zip(row.tolist(), col.tolist(), (sign < 0).astype(int).tolist(), hmat[a, b].tolist()))


@pytest.mark.parametrize("which", ["2x4", "2x2+bath", "4x4", "dense7"])
def test_hop_table_bit_exact(which):
    if which == "2x4":
        c = W.plain_2x4()
    elif which == "2x2+bath":
        c = W.cdmft_2x2_bath()
    elif which == "4x4":
        c = W.periodic_4x4()
    else:
        c = W.random_cluster(np.random.default_rng(7), 5, 2, 3, 2, dense_t=True)
    m = _model(c)
    with ed.Cluster(c) as cl:
        for N in sorted({c["n_up"], c["n_up"] + 1, c["n_up"] - 1, 1, m.L - 1}):
            if 0 <= N <= m.L:
                assert _gpu_table_tuples(cl.h, N, m.L) == _oracle_table_tuples(m.h, N)


# ------------------------------------------------------------------ K3: H.psi
def _hpsi_gpu(cl, nu, nd, psi, dtype):
    tdt = torch.float64 if dtype == ed.ED_FP64 else torch.float32
    x = torch.tensor(psi, dtype=tdt, device="cuda")
    y = torch.full_like(x, float("nan"))
    ed.ed_hpsi(cl.h, nu, nd, dtype, x.data_ptr(), y.data_ptr(), 0, _stream())
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


SMALL = [("2x4", W.plain_2x4()),
         ("2x2+bath", W.cdmft_2x2_bath()),
         ("rand-bath", W.random_cluster(np.random.default_rng(3), 3, 3, 2, 4)),
         ("chain5", W.random_cluster(np.random.default_rng(4), 5, 0, 1, 4))]


@pytest.mark.parametrize("name,c", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("shift", [(0, 0), (1, 0), (-1, 0), (0, 1)])
def test_hpsi_matches_oracle(name, c, shift):
    m = _model(c)
    nu, nd = c["n_up"] + shift[0], c["n_dn"] + shift[1]
    if not (0 <= nu <= m.L and 0 <= nd <= m.L):
        pytest.skip("sector does not exist")
    op = O.sector_hamiltonian(m, nu, nd)
    psi = np.random.default_rng(11).standard_normal(op.shape2)
    ref = O.apply_h(op, psi)
    with ed.Cluster(c) as cl:
        y64 = _hpsi_gpu(cl, nu, nd, psi, ed.ED_FP64)
        y32 = _hpsi_gpu(cl, nu, nd, psi.astype(np.float32), ed.ED_FP32)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(y64 - ref)) <= 1e-12 * scale
    ref32 = O.apply_h(op, psi.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(y32 - ref32)) <= 2e-5 * scale


def test_hpsi_full_size_sampled():
    """4x4 periodic half filling (d = 165,636,900), in the launch configuration the benchmark
    uses: sampled elements of y = H x, each computed one by one by the oracle."""
    c = W.periodic_4x4()
    op = O.sector_hamiltonian(_model(c), 8, 8)
    du, dd = op.shape2
    rng = np.random.default_rng(5)
    us = np.concatenate([[0, du - 1, 0, du - 1], rng.integers(0, du, 2000)])
    ds = np.concatenate([[0, dd - 1, dd - 1, 0], rng.integers(0, dd, 2000)])
    with ed.Cluster(c) as cl:
        for dtype, tdt in ((ed.ED_FP32, torch.float32), (ed.ED_FP64, torch.float64)):
            g = torch.Generator(device="cuda")
            g.manual_seed(9)
            x = torch.rand((du, dd), generator=g, device="cuda", dtype=tdt) * 2 - 1
            y = torch.empty_like(x)
            ed.ed_hpsi(cl.h, 8, 8, dtype, x.data_ptr(), y.data_ptr(), 0, _stream())
            torch.cuda.synchronize()
            ysel = y[torch.as_tensor(us, device="cuda"), torch.as_tensor(ds, device="cuda")].double().cpu().numpy()
            psi = x.cpu().numpy().astype(np.float64)
            del x, y
            torch.cuda.empty_cache()
            ref = O.apply_h_sampled(op, psi, us, ds)
            del psi
            tol = 1e-12 if dtype == ed.ED_FP64 else 2e-5
            assert np.max(np.abs(ysel - ref)) <= tol * np.max(np.abs(ref))


# ------------------------------------------------------------------ ground state
def test_ground_state_2x4():
    c = W.plain_2x4()
    m = _model(c)
    E0, Om, gap = O.ground_state(O.sector_hamiltonian(m, 4, 4))
    with ed.Cluster(c) as cl:
        st, E, res, it = cl.ground_state()
        assert st == ed.ED_OK
        assert abs(E - E0) <= 1e-10 * abs(E0)
        assert res <= 1e-12
        W_ = cl.ground_vector()
    assert abs(abs(np.vdot(W_, Om)) - 1.0) < 1e-10


@pytest.mark.parametrize("t,U,mu", [(-1.0, 4.0, 0.0), (0.7, 2.5, 1.3)])
def test_ground_state_dimer_closed_form(t, U, mu):
    c = W.hubbard_dimer(t, U, mu)
    with ed.Cluster(c) as cl:
        st, E, res, it = cl.ground_state()
    assert E == pytest.approx(0.5 * (U - math.sqrt(U * U + 16 * t * t)) - 2 * mu, abs=1e-12)


def test_ground_state_free_fermions():
    c = W.random_cluster(np.random.default_rng(12), 6, 2, 3, 5, U=0.0)
    eps = np.linalg.eigvalsh(_model(c).h)
    with ed.Cluster(c) as cl:
        st, E, res, it = cl.ground_state()
    assert E == pytest.approx(eps[:3].sum() + eps[:5].sum(), abs=1e-11)


@pytest.mark.parametrize("precision", [ed.ED_FP64, ed.ED_FP32])
def test_ground_state_cdmft_impurity(precision):
    """2x2 plaquette + 8 bath orbitals, d = 853,776: FP64 and FP32-storage forms, E0 to 1e-10."""
    c = W.cdmft_2x2_bath()
    E0, _, _ = O.ground_state(O.sector_hamiltonian(_model(c), 6, 6))
    with ed.Cluster(c, precision=precision) as cl:
        st, E, res, it = cl.ground_state()
    assert st in (ed.ED_OK, ed.ED_WARN_DEGENERATE)
    assert abs(E - E0) <= 1e-10 * abs(E0)


# ------------------------------------------------------------------ Green function
def test_green_2x4_continued_fraction():
    """2x4 open, U = 4, half filling: all 8 x 8 G_ij on 1000 real frequencies, eta = 0.05."""
    c = W.plain_2x4()
    om = W.real_grid(1000)
    z = om + 0.05j
    Gref = O.green_exact(_model(c), 4, 4, z)[0]
    with ed.Cluster(c) as cl:
        st, G = ed.ed_green(cl.h, om, 0.05, 8)
    assert np.max(np.abs(G - Gref)) <= 1e-8


GF_CASES = [("bath-asym", W.random_cluster(np.random.default_rng(21), 3, 3, 2, 4), 0),
            ("bath-down", W.random_cluster(np.random.default_rng(22), 3, 2, 3, 2), 1),
            ("chain-low", W.random_cluster(np.random.default_rng(23), 6, 0, 1, 2), 0),
            ("nearly-full", W.random_cluster(np.random.default_rng(24), 4, 1, 5, 3), 0),
            ("one-site", W._cluster("atom", np.zeros((1, 1)), 5.0, 1.5, 1, 1), 0)]


@pytest.mark.parametrize("name,c,spin", GF_CASES, ids=[g[0] for g in GF_CASES])
@pytest.mark.parametrize("axis", [ed.ED_AXIS_REAL, ed.ED_AXIS_MATSUBARA])
def test_green_matches_exact(name, c, spin, axis):
    m = _model(c)
    if axis == ed.ED_AXIS_REAL:
        om = W.real_grid(301)
        z = om + 0.05j
    else:
        om = W.matsubara_grid(256, 50.0)
        z = 1j * om
    Gref, Q, w, E0, gap = O.green_exact(m, c["n_up"], c["n_dn"], z, spin=spin)
    with ed.Cluster(c) as cl:
        st, G = ed.ed_green(cl.h, om, 0.05, m.ns, axis=axis, spin=spin)
    assert np.max(np.abs(G - Gref)) <= 1e-8
