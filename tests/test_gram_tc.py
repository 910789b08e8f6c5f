"""The Gram kernels of the band Lanczos orthogonalization (Sec. 4.4) on random FP32 vectors:
the tensor-core kernel (tcgen05 MMA, 3xTF32 split, TMA loads) and the CUDA-core one against the
FP64 product of the same FP32 values computed on the host.

Bound: every product of the 3xTF32 split carries a relative error <= 2^-21 (the low part keeps 13
bits of which TF32 holds 11), sums run in FP32 over at most 16 x 32 elements, then in FP64; so
|G - G_exact| <= 4 * 2^-21 * sum_e |x_e y_e| + a few FP32 roundings of partial sums.  Asserted:
1e-6 * sum_e |x_e y_e| per entry (about 2x the product bound)."""

import numpy as np
import pytest

from paper_2305_18643_gb300 import build, ed

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def libed():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return ed.lib()


def _vectors(nv, n, vstride, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    V = torch.zeros((nv, vstride), dtype=torch.float32, device="cuda")
    V[:, :n] = torch.randn((nv, n), generator=g, device="cuda", dtype=torch.float32)
    return V


def _check(V, nx, Yv, ny, n, vstride, method, sym=False):
    G = ed.ed_gram_f32(V.data_ptr(), nx, Yv.data_ptr(), ny, vstride, n, method)
    X = V[:nx, :n].double()
    Y = Yv[:ny, :n].double()
    ref = (X @ Y.T).cpu().numpy()
    scale = (X.abs() @ Y.abs().T).cpu().numpy()
    err = np.abs(G - ref)
    assert np.all(err <= 1e-6 * scale + 1e-12), float((err / scale).max())
    return G


@pytest.mark.parametrize("n,vstride", [(32 * 1000, 32 * 1000), (32 * 12345, 32 * 12345 + 96), (4096, 4224)])
@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 16), (8, 8), (16, 5)], ids=["16x16", "32x16", "8x8", "16x5"])
def test_tensor_core_gram_matches_fp64(n, vstride, nx, ny):
    """Two X blocks (32 x 16, the projection on X_{j-1}, X_j), one block, partial blocks whose
    rows past the vectors must read as zero, element counts below and above one tile per CTA."""
    V = _vectors(nx + ny, n, vstride, seed=nx * 100 + ny)
    Y = V[nx:]
    G1 = _check(V, nx, Y, ny, n, vstride, 1)
    G0 = _check(V, nx, Y, ny, n, vstride, 0)
    assert G1.shape == G0.shape


@pytest.mark.parametrize("nx", [16, 11])
def test_tensor_core_gram_symmetric(nx):
    """W^T W (X == Y): the symmetric form."""
    n, vstride = 32 * 5000, 32 * 5000
    V = _vectors(nx, n, vstride, seed=nx)
    G = _check(V, nx, V, nx, n, vstride, 1, sym=True)
    assert np.max(np.abs(G - G.T)) <= 1e-6 * np.max(np.abs(G))


def test_tensor_core_gram_full_band_size():
    """The size of a band block step at the 4x4 cluster: 48 vectors of 147,232,800 elements
    (rows padded to 12,928: 147,896,320 stored), the projection [X_{j-1}, X_j]^T W and W^T W, and
    repeated calls give identical results (fixed reduction order)."""
    n = 11440 * 12928
    V = _vectors(48, n, n, seed=7)
    W = V[32:]
    G1 = _check(V, 32, W, 16, n, n, 1)
    G2 = ed.ed_gram_f32(V.data_ptr(), 32, W.data_ptr(), 16, n, n, 1)
    assert np.array_equal(G1, G2)
    _check(W, 16, W, 16, n, n, 1, sym=True)
    del V, W
    torch.cuda.empty_cache()


def test_tensor_core_gram_rejects_unaligned_layouts():
    V = _vectors(17, 4096, 4096, seed=1)
    with pytest.raises(ed.EDError) as e:
        ed.ed_gram_f32(V.data_ptr(), 16, V[16:].data_ptr(), 1, 4096, 4000, 1)  # n not a multiple of 32
    assert e.value.status == ed.ED_ERR_INVALID
