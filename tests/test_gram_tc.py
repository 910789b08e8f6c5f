"""The Gram kernels of the band Lanczos orthogonalization (Sec. 4.4) on random FP32 vectors:
the tensor-core kernel (tcgen05 MMA on TF32 head/tail splits, TMA loads) and the CUDA-core one
against the FP64 product of the same FP32 values computed on the host.

Bound: with x = h + l + r, h and l TF32 rounded to nearest, |r| <= 2^-22 |x|, so every product
x y is carried by h h' + h l' + l h' + l l' to within 2^-21 |x y|; those four products are exact
in FP32 and each sits in its own TMEM accumulator for four MMAs (8 elements each), then in a
compensated FP32 sum, then FP64.  Worst case per entry about 2^-20 sum_e |x_e y_e|; the
rounding errors are unbiased, so the observed error is far below it.  Asserted: 1e-6 sum_e |x_e y_e|
per entry.  A shared accumulator over many MMAs (the kernel's first form) gave a one-sided
1e-5 on the diagonal of W^T W, which the symmetric test catches."""

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
    """n not a multiple of 32 (a K-tile), or a vector stride that is not a multiple of 16 bytes
    (a TMA row stride), is refused before any launch."""
    V = _vectors(17, 4096, 4096, seed=1)
    for vstride, n in ((4096, 4004), (4098, 4000)):
        with pytest.raises(ed.EDError) as e:
            ed.ed_gram_f32(V.data_ptr(), 16, V[16:].data_ptr(), 1, vstride, n, 1)
        assert e.value.status == ed.ED_ERR_INVALID
