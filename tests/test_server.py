"""Served form on the GPU: requests of different sizes solved side by side give the same results
as alone and as the oracle; admission by memory; bounded waits, cancellation and a failure made
on the host (the test hook), with the server still serving the other requests."""

import numpy as np
import pytest

import oracle as O
import oracle_memo as OM
from paper_2305_18643_gb300 import build, ed
from paper_2305_18643_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def libed():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return ed.lib()


def _model(c):
    return O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])


def _mix():
    """Requests taking both paths: 2x2 + 2 bath and 2x3 (batched path: sectors <= 100000) and
    the 12-orbital impurity (single-cluster path)."""
    rng = np.random.default_rng(20230529 + 5000)
    small = [W.random_cluster(rng, 4, 2, 3, 3), W.random_cluster(rng, 3, 3, 2, 4),
             W.served_request(rng, sizes=(6,)), W.served_request(rng, sizes=(8,))]
    return small + [W.cdmft_2x2_bath()]


def _submit_all(srv, clusters, om, axis, precision):
    return [srv.submit(c, omega=om, eta=0.05, axis=axis, precision=precision, seed=11 + k, cf_max_levels=2000)
            for k, c in enumerate(clusters)]


@pytest.mark.parametrize("precision", [ed.ED_FP64, ed.ED_FP32], ids=["fp64", "fp32"])
def test_served_same_alone_and_in_the_mix(precision):
    """Every request gives the same E0 and G when it is solved alone (a server with one lane and
    nothing else queued) and among the others (three lanes, all submitted at once)."""
    clusters = _mix()
    om = W.matsubara_grid(128)
    with ed.Server(16 * GB, max_slots=3, paused=1) as srv:
        ids = _submit_all(srv, clusters, om, ed.ED_AXIS_MATSUBARA, precision)
        srv.pause(False)
        mixed = [srv.wait(i) for i in ids]
        stats = srv.stats()
    assert stats["completed"] == len(clusters) and stats["failed"] == 0
    assert stats["batched_solves"] >= 1
    paths = [r["path"] for r, _ in mixed]
    assert paths[-1] == 0 and all(p == 1 for p in paths[:-1])
    assert all(r["batch_size"] == len(clusters) - 1 for r, _ in mixed[:-1])
    for k, c in enumerate(clusters):
        with ed.Server(16 * GB, max_slots=1) as srv:
            rid = srv.submit(c, omega=om, eta=0.05, axis=ed.ED_AXIS_MATSUBARA, precision=precision, seed=11 + k,
                             cf_max_levels=2000)
            alone, Ga = srv.wait(rid)
        rm, Gm = mixed[k]
        assert alone["batch_size"] == 1 and alone["path"] == rm["path"]
        assert rm["status"] >= 0 and alone["status"] == rm["status"]
        assert abs(alone["E0"] - rm["E0"]) <= 1e-12 * max(1.0, abs(rm["E0"])), k
        assert np.max(np.abs(Ga - Gm)) <= 1e-10, k


def test_served_results_match_the_oracle():
    """FP64 requests through the server: E0 to 1e-10 and G of both spins to 1e-8 of the exact
    Lehmann sum (clusters of <= 8 orbitals)."""
    rng = np.random.default_rng(20230529 + 5001)
    clusters = [W.random_cluster(rng, 4, 2, 3, 2), W.served_request(rng, sizes=(8,)), W.random_cluster(rng, 3, 3, 4, 3)]
    om = W.real_grid(101)
    with ed.Server(8 * GB, max_slots=2, batch_max_dim=3000) as srv:  # the 2x4 cluster takes the single path
        ids = [srv.submit(c, omega=om, eta=0.05, precision=ed.ED_FP64, seed=5 + k, cf_max_levels=20000)
               for k, c in enumerate(clusters)]
        out = [srv.wait(i) for i in ids]
    assert {r["path"] for r, _ in out} == {0, 1}
    for (r, G), c in zip(out, clusters):
        m = _model(c)
        for spin in (0, 1):
            Gx, _, _, E0, gap = OM.green_exact(m, c["n_up"], c["n_dn"], om + 0.05j, spin=spin)
            assert abs(r["E0"] - E0) <= 1e-10 * max(1.0, abs(E0))
            if gap > 1e-6:
                assert np.max(np.abs(G[spin] - Gx)) <= 1e-8


def test_admission_by_memory():
    """A budget that holds one 12-orbital request at a time: they run one after another (never
    two at once) and all complete; a request larger than the whole budget is refused at submit."""
    c = W.cdmft_2x2_bath()
    one = ed.ed_request_bytes(c, n_freq=64, precision=ed.ED_FP32)
    budget = int(one * 1.5)
    om = W.matsubara_grid(64)
    with ed.Server(budget, max_slots=4) as srv:
        ids = [srv.submit(c, omega=om, axis=ed.ED_AXIS_MATSUBARA, precision=ed.ED_FP32, seed=k) for k in range(3)]
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
        assert st["max_running"] == 1 and st["completed"] == 3
        assert st["peak_reserved_bytes"] <= budget
        with pytest.raises(ed.EDError) as e:
            srv.submit(W.periodic_4x4(), omega=om, axis=ed.ED_AXIS_MATSUBARA, precision=ed.ED_FP32)
        assert e.value.status == ed.ED_ERR_TOO_LARGE
    E = [r["E0"] for r, _ in res]
    assert max(E) - min(E) <= 1e-9 * abs(E[0])  # the same cluster, seeds differ


def test_requests_overlap_on_the_device():
    """With room for several, requests of the single-cluster path run at the same time."""
    c = W.cdmft_2x2_bath()
    om = W.matsubara_grid(64)
    with ed.Server(64 * GB, max_slots=4, paused=1) as srv:
        ids = [srv.submit(c, omega=om, axis=ed.ED_AXIS_MATSUBARA, precision=ed.ED_FP32, seed=k) for k in range(4)]
        srv.pause(False)
        for i in ids:
            srv.wait(i)
        assert srv.stats()["max_running"] >= 2


def test_wait_timeout_cancel_and_host_failure():
    """Requests queued behind a paused admission: ed_wait with a zero timeout reports
    ED_ERR_TIMEOUT; a queued request is cancelled; a failure injected on the host ends one
    request with that status; the requests around them complete normally."""
    big = W.cdmft_2x2_bath()
    small = W.plain_2x4()
    om = W.real_grid(256)
    with ed.Server(16 * GB, max_slots=1, batch_max_dim=0, paused=1) as srv:
        r_big = srv.submit(big, omega=om, precision=ed.ED_FP64, seed=1)
        r_cancel = srv.submit(small, omega=om, precision=ed.ED_FP64, seed=2)
        r_fail = srv.submit(small, omega=om, precision=ed.ED_FP64, seed=3)
        r_ok = srv.submit(small, omega=om, precision=ed.ED_FP64, seed=4, cf_max_levels=20000)
        with pytest.raises(ed.EDError) as e:
            srv.wait(r_big, timeout_s=0.0)
        assert e.value.status == ed.ED_ERR_TIMEOUT
        srv.cancel(r_cancel)
        srv.inject_failure(r_fail, ed.ED_ERR_CUDA)
        srv.pause(False)
        rb, _ = srv.wait(r_big)
        rc, _ = srv.wait(r_cancel)
        rf, _ = srv.wait(r_fail)
        ro, Go = srv.wait(r_ok)
        st = srv.stats()
        with pytest.raises(ed.EDError) as e:
            srv.poll(r_ok)  # collected already
        assert e.value.status == ed.ED_ERR_NOT_FOUND
    assert rb["status"] >= 0 and ro["status"] >= 0
    assert rc["status"] == ed.ED_ERR_CANCELLED
    assert rf["status"] == ed.ED_ERR_CUDA
    assert st["failed"] == 1 and st["cancelled"] == 1 and st["completed"] == 2
    m = _model(small)
    Gx, _, _, E0, _ = OM.green_exact(m, 4, 4, om + 0.05j, spin=0)
    assert abs(ro["E0"] - E0) <= 1e-10 * abs(E0)
    assert np.max(np.abs(Go[0] - Gx)) <= 1e-8


def test_destroy_with_work_in_flight():
    """Destroying a server with running and queued requests returns (they are cancelled)."""
    c = W.cdmft_2x2_bath()
    srv = ed.Server(16 * GB, max_slots=1, batch_max_dim=0)
    for k in range(3):
        srv.submit(c, omega=W.real_grid(64), precision=ed.ED_FP64, seed=k)
    srv.close()


def test_concurrent_band_requests_of_different_sizes():
    """Band requests of 12 and 14 orbitals on concurrent lanes (their kernels launch with different
    shared-memory sizes at the same time) all complete, with the energies of the same requests
    solved alone."""
    rng = np.random.default_rng(20230529 + 5002)
    reqs = [W.served_request(rng, sizes=(n,)) for n in (12, 14, 12, 14, 12, 14)]
    om = W.matsubara_grid(256)
    with ed.Server(64 * GB, max_slots=6, batch_max_dim=0, paused=1) as srv:
        ids = [srv.submit(c, omega=om, axis=ed.ED_AXIS_MATSUBARA, precision=ed.ED_FP32, gf_method=ed.ED_GF_BAND,
                          seed=3 + k) for k, c in enumerate(reqs)]
        srv.pause(False)
        out = [srv.wait(i)[0] for i in ids]
        assert srv.stats()["max_running"] >= 2
    for r in out:
        assert r["status"] >= 0, r.get("error")
    with ed.Server(64 * GB, max_slots=1, batch_max_dim=0) as srv:
        for k in (0, 1):
            alone = srv.wait(srv.submit(reqs[k], omega=om, axis=ed.ED_AXIS_MATSUBARA, precision=ed.ED_FP32,
                                        gf_method=ed.ED_GF_BAND, seed=3 + k))[0]
            assert abs(alone["E0"] - out[k]["E0"]) <= 1e-12 * abs(alone["E0"])


def test_served_14_orbital_band_request_matches_the_oracle():
    """A served band request of 14 orbitals (FP64, the two-pass kernels on a lane): its ground
    energy equals the oracle's (tests/golden/ladder14_band.npz) to 1e-10, and its G equals what
    the single-cluster path gives for the same cluster (the path whose band G is compared with
    the oracle's band Lanczos in tests/test_benchmarked_paths.py)."""
    import os
    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ladder14_band.npz"))
    c = W.served_request(np.random.default_rng(int(g["seed"])), sizes=(14,))
    om = W.matsubara_grid(64)
    with ed.Server(64 * GB, max_slots=2, batch_max_dim=0) as srv:
        r, G = srv.wait(srv.submit(c, omega=om, axis=ed.ED_AXIS_MATSUBARA, precision=ed.ED_FP64,
                                   gf_method=ed.ED_GF_BAND, seed=11))
    assert r["status"] >= 0, r.get("error")
    assert abs(r["E0"] - float(g["E0"])) <= 1e-10 * abs(float(g["E0"]))
    with ed.Cluster(c, precision=ed.ED_FP64, gf_method=ed.ED_GF_BAND, seed=11) as cl:
        st, Gs = ed.ed_green(cl.h, om, 0.0, 14, axis=ed.ED_AXIS_MATSUBARA)
    assert np.max(np.abs(G[0] - Gs)) <= 1e-10
