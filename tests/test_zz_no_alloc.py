"""ed_hpsi_dots_static, the entry point for callers that cannot allocate device memory (their
GPU memory is managed by their own pool or caching allocator): its product must equal the one
of ed_hpsi and its three reductions the dot products of that product, on two calls in a row
(the fixed scratch array is shared by every call and keeps the previous call's contents).

This file is collected last so that a run stopping at the first failure has run every other
test first."""

import numpy as np
import pytest

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


@pytest.mark.parametrize("name,c", CASES, ids=[x[0] for x in CASES])
@pytest.mark.parametrize("dtype", [ed.ED_FP64, ed.ED_FP32], ids=["fp64", "fp32"])
def test_static_scratch_matches_hpsi(name, c, dtype):
    tdt = torch.float64 if dtype == ed.ED_FP64 else torch.float32
    tol = 1e-12 if dtype == ed.ED_FP64 else 2e-5
    stream = torch.cuda.current_stream().cuda_stream
    with ed.Cluster(c) as cl:
        du, dd = ed.ed_sector_dims(cl.h, c["n_up"], c["n_dn"])
        g = torch.Generator(device="cuda")
        g.manual_seed(3)
        for call in range(2):
            x = (torch.rand((du, dd), generator=g, device="cuda", dtype=torch.float64) * 2 - 1).to(tdt)
            y_ref = torch.full_like(x, float("nan"))
            ed.ed_hpsi(cl.h, c["n_up"], c["n_dn"], dtype, x.data_ptr(), y_ref.data_ptr(), 0, stream)
            y = torch.full_like(x, float("nan"))
            out3 = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            ed.ed_hpsi_dots_static(cl.h, dtype, x.data_ptr(), y.data_ptr(), out3.data_ptr(), 0, stream)
            torch.cuda.synchronize()
            scale = float(y_ref.abs().max())
            assert float((y - y_ref).abs().max()) <= tol * scale
            xd, yd = x.double(), y_ref.double()
            ref = torch.stack([(xd * yd).sum(), (yd * yd).sum(), (xd * xd).sum()]).cpu().numpy()
            got = out3.cpu().numpy()
            assert np.all(np.abs(got - ref) <= tol * np.abs(ref) + 1e-12), (call, got, ref)


def test_static_scratch_rejects_large_sectors():
    """The 4x4 half-filled sector (1.66e8 elements) exceeds the 4,194,304 elements of the fixed
    scratch: rejected with ED_ERR_TOO_LARGE before any launch."""
    with ed.Cluster(W.periodic_4x4()) as cl:
        with pytest.raises(ed.EDError) as err:
            ed.ed_hpsi_dots_static(cl.h, ed.ED_FP32, 16, 16, 16)
        assert err.value.status == ed.ED_ERR_TOO_LARGE
