"""ed_hpsi_dots_static, the entry point for callers that cannot allocate device memory (their
GPU memory is managed by their own pool or caching allocator): its product must equal the one
of ed_hpsi and of the CPU oracle, and its three reductions the dot products of that product,
on two calls in a row (the fixed scratch array is shared by every call and keeps the previous
call's contents).

This file is collected last so that a run stopping at the first failure has run every other
test first."""

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


CASES = [("2x2+bath", W.cdmft_2x2_bath()), ("2x4", W.plain_2x4()),
         ("bath-asym", W.random_cluster(np.random.default_rng(21), 3, 3, 2, 4))]


def _model(c):
    return O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])


@pytest.mark.parametrize("name,c", CASES, ids=[x[0] for x in CASES])
@pytest.mark.parametrize("dtype", [ed.ED_FP64, ed.ED_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("pad", [0, 5], ids=["ld=d_dn", "ld=d_dn+5"])
def test_static_scratch_matches_hpsi(name, c, dtype, pad):
    """Two calls in a row with different inputs; rows padded by `pad` elements whose contents
    must stay untouched (NaN in, NaN out)."""
    tdt = torch.float64 if dtype == ed.ED_FP64 else torch.float32
    tol = 1e-12 if dtype == ed.ED_FP64 else 2e-5
    stream = torch.cuda.current_stream().cuda_stream
    op = O.sector_hamiltonian(_model(c), c["n_up"], c["n_dn"])
    with ed.Cluster(c) as cl:
        du, dd = ed.ed_sector_dims(cl.h, c["n_up"], c["n_dn"])
        ld = dd + pad
        rng = np.random.default_rng(3)
        for call in range(2):
            psi = rng.uniform(-1.0, 1.0, (du, dd))
            x = torch.full((du, ld), float("nan"), dtype=tdt, device="cuda")
            x[:, :dd] = torch.as_tensor(psi, device="cuda").to(tdt)
            y_ref = torch.full_like(x, float("nan"))
            ed.ed_hpsi(cl.h, c["n_up"], c["n_dn"], dtype, x.data_ptr(), y_ref.data_ptr(), ld if pad else 0, stream)
            y = torch.full_like(x, float("nan"))
            out3 = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            ed.ed_hpsi_dots_static(cl.h, dtype, x.data_ptr(), y.data_ptr(), out3.data_ptr(), ld if pad else 0, stream)
            torch.cuda.synchronize()
            if pad:
                assert bool(torch.isnan(y[:, dd:]).all()), "padding written"
            yv, yr = y[:, :dd].double().cpu().numpy(), y_ref[:, :dd].double().cpu().numpy()
            # the oracle's product of the same (rounded) input
            ref = O.apply_h(op, x[:, :dd].double().cpu().numpy())
            scale = float(np.max(np.abs(ref)))
            assert float(np.max(np.abs(yv - ref))) <= tol * scale, call
            assert float(np.max(np.abs(yv - yr))) <= tol * scale, call
            xd = x[:, :dd].double().cpu().numpy()
            want = np.array([np.sum(xd * ref), np.sum(ref * ref), np.sum(xd * xd)])
            got = out3.cpu().numpy()
            assert np.all(np.abs(got - want) <= 10 * tol * np.abs(want) + 1e-12), (call, got, want)


def test_static_scratch_rejects_large_sectors():
    """A 2x7 half-filled cluster (3432^2 = 11,778,624 elements) exceeds the 4,194,304 elements of
    the fixed scratch: rejected with ED_ERR_TOO_LARGE before any launch.  The buffers are real
    and of full size, so even if the size check were lost the kernel would stay inside them."""
    c = W.served_request(np.random.default_rng(4), sizes=(14,))
    with ed.Cluster(c) as cl:
        du, dd = ed.ed_sector_dims(cl.h, c["n_up"], c["n_dn"])
        assert du * dd > 4194304
        x = torch.zeros((du, dd), dtype=torch.float32, device="cuda")
        y = torch.full_like(x, float("nan"))
        out3 = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        with pytest.raises(ed.EDError) as err:
            ed.ed_hpsi_dots_static(cl.h, ed.ED_FP32, x.data_ptr(), y.data_ptr(), out3.data_ptr())
        assert err.value.status == ed.ED_ERR_TOO_LARGE
        torch.cuda.synchronize()
        assert bool(torch.isnan(y).all()) and bool(torch.isnan(out3).all())


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs a second GPU to make the current device differ from the cluster's")
def test_static_scratch_rejects_other_device():
    """A cluster built on device 0 called while device 1 is current: rejected before any launch
    (the tables are on device 0, the scratch and the caller's buffers on device 1)."""
    c = W.plain_2x4()
    with ed.Cluster(c) as cl:
        with torch.cuda.device(1):
            x = torch.zeros((70, 70), dtype=torch.float64, device="cuda:1")
            y = torch.zeros_like(x)
            out3 = torch.zeros(3, dtype=torch.float64, device="cuda:1")
            with pytest.raises(ed.EDError) as err:
                ed.ed_hpsi_dots_static(cl.h, ed.ED_FP64, x.data_ptr(), y.data_ptr(), out3.data_ptr())
            assert err.value.status == ed.ED_ERR_INVALID
