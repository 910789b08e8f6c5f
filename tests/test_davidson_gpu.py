"""Parity of the Davidson low states and of the mixed-state Green function (the paper's
recommendation for degenerate ground states, Sec. 4.2, and the Davidson_states / temperature
options of Sec. 9) with the oracle: energies to 1e-10 relative, G to 1e-8 absolute."""

import math

import numpy as np
import pytest

import oracle as O
import oracle_memo as OM
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


def _ring(n_up, n_dn, U=2.5, t=-1.0):
    T = W.lattice_hopping(4, 1, t=t, periodic=True)
    return W._cluster("4-ring", T, U, 0.3, n_up, n_dn)


def test_dimer_four_states_closed_form():
    """All four states of the half-filled dimer: (U -+ sqrt(U^2 + 16 t^2)) / 2, 0, U, less 2 mu."""
    t, U, mu = -1.0, 4.0, 0.5
    c = W.hubbard_dimer(t, U, mu)
    with ed.Cluster(c) as cl:
        ed.ed_set_option(cl.h, ed.ED_OPT_DAVIDSON_STATES, 4)
        st, E0, res, it = cl.ground_state()
        E, wt = ed.ed_low_states(cl.h)
    r = math.sqrt(U * U + 16 * t * t)
    want = np.sort([(U - r) / 2, 0.0, U, (U + r) / 2]) - 2 * mu
    assert np.allclose(E, want, atol=1e-12)
    assert np.allclose(wt, [1, 0, 0, 0])
    assert res <= 1e-12


@pytest.mark.parametrize("method", [ed.ED_GF_CF, ed.ED_GF_BAND], ids=["cf", "band"])
@pytest.mark.parametrize("T", [0.0, 0.4], ids=["T=0", "T=0.4"])
def test_degenerate_ring_mixed_green(method, T):
    """4-site ring, N_up = 2, N_dn = 1, U = 2.5: a doubly degenerate ground state.  Lanczos alone
    flags it (G not unique); with three Davidson states the mixed-state G equals the oracle's on the
    real and Matsubara axes (equal weights at T = 0, Boltzmann weights at T = 0.4)."""
    c = _ring(2, 1)
    m = _model(c)
    for axis in (ed.ED_AXIS_REAL, ed.ED_AXIS_MATSUBARA):
        om = W.real_grid(201) if axis == ed.ED_AXIS_REAL else W.matsubara_grid(128, 50.0)
        z = om + 0.05j if axis == ed.ED_AXIS_REAL else 1j * om
        Gref, Eref, pref = O.green_mixed(m, 2, 1, z, k=3, T=T)
        assert abs(Eref[1] - Eref[0]) < 1e-10
        with ed.Cluster(c, gf_method=method) as cl:
            ed.ed_set_option(cl.h, ed.ED_OPT_DAVIDSON_STATES, 3)
            ed.ed_set_option(cl.h, ed.ED_OPT_TEMPERATURE, T)
            st, E0, res, it = cl.ground_state()
            E, wt = ed.ed_low_states(cl.h)
            stg, G = ed.ed_green(cl.h, om, 0.05, 4, axis=axis)
        assert st == ed.ED_OK  # a state above the degenerate pair was found
        assert np.allclose(E, Eref, rtol=0, atol=1e-10 * max(1.0, abs(Eref[0])))
        assert np.allclose(wt, pref, atol=1e-10)
        assert np.max(np.abs(G - Gref)) <= 1e-8


@pytest.mark.parametrize("name,c,k", [
    ("bath-asym", W.random_cluster(np.random.default_rng(21), 3, 3, 2, 4), 4),
    ("2x4", W.plain_2x4(), 5),
    ("2x2+bath", W.cdmft_2x2_bath(), 3)], ids=["bath-asym", "2x4", "2x2+bath"])
def test_low_states_match_oracle(name, c, k):
    """k lowest energies of sectors of 350 to 853,776 states against the oracle (LAPACK / ARPACK)
    to 1e-10 relative, residuals to 1e-12; the 12-orbital sector takes the two-pass H.psi when
    forced (ED_OPT_TWO_PASS_MIN_BYTES = 0)."""
    m = _model(c)
    with OM.dense_blas_threads():
        Eref, V = O.low_states(O.sector_hamiltonian(m, c["n_up"], c["n_dn"]), k)
    with ed.Cluster(c) as cl:
        if name == "2x2+bath":
            ed.ed_set_option(cl.h, ed.ED_OPT_TWO_PASS_MIN_BYTES, 0)
        ed.ed_set_option(cl.h, ed.ED_OPT_DAVIDSON_STATES, k)
        st, E0, res, it = cl.ground_state()
        E, wt = ed.ed_low_states(cl.h)
        Wv = cl.ground_vector()
    assert st in (ed.ED_OK, ed.ED_WARN_DEGENERATE)
    assert np.allclose(E, Eref, rtol=0, atol=1e-10 * max(1.0, abs(Eref[0])))
    assert res <= 1e-12
    assert abs(abs(np.vdot(Wv, V[0])) - 1.0) < 1e-8 or abs(Eref[1] - Eref[0]) < 1e-8
