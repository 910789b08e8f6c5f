"""Host-side logic of the served form that needs no GPU: the device footprint used for admission
(closed forms of the sector dimensions, no CUDA call) and argument checking."""

import math

import numpy as np
import pytest

from paper_2305_18643_gb300 import ed
from paper_2305_18643_gb300 import workloads as W


def test_footprint_covers_ground_state_vectors():
    """At least the FP64 ground state, the FP64 polish vector and three padded Lanczos vectors."""
    c = W.cdmft_2x2_bath()
    d = math.comb(12, 6) ** 2
    ld = (math.comb(12, 6) + 127) // 128 * 128
    b = ed.ed_request_bytes(c, n_freq=0)
    assert b >= d * 16 + 3 * math.comb(12, 6) * ld * 8


def test_footprint_grows_with_the_green_function():
    c = W.plain_2x4()
    b0 = ed.ed_request_bytes(c, n_freq=0)
    b1 = ed.ed_request_bytes(c, n_freq=100)
    b2 = ed.ed_request_bytes(c, n_freq=1000)
    assert b0 < b1 < b2
    # G of both spins, complex128: 2 x n_freq x 8 x 8 x 16 bytes at least
    assert b2 - b0 >= 2 * 1000 * 64 * 16


def test_footprint_fp32_not_larger_and_budget_caps_vectors():
    c = W.cdmft_2x2_bath()
    f64 = ed.ed_request_bytes(c, n_freq=512, precision=ed.ED_FP64)
    f32 = ed.ed_request_bytes(c, n_freq=512, precision=ed.ED_FP32)
    assert f32 <= f64
    # with a small Green-function budget only 2 vectors of the largest N+-1 sector are reserved
    small = ed.ed_request_bytes(c, n_freq=512, precision=ed.ED_FP64, gf_budget=1)
    big = ed.ed_request_bytes(c, n_freq=512, precision=ed.ED_FP64, gf_budget=0)
    dt = math.comb(12, 7) * ((math.comb(12, 6) + 127) // 128 * 128)
    assert small < big
    assert big - small >= (4 + 6 - 2) * 2 * dt * 8  # R = 4 + 6 runs of 2 vectors, less the 2 kept


def test_footprint_band_ring_vs_full():
    c = W.cdmft_2x2_bath()
    ring = ed.ed_request_bytes(c, n_freq=64, gf_method=ed.ED_GF_BAND, gf_budget=1)
    full = ed.ed_request_bytes(c, n_freq=64, gf_method=ed.ED_GF_BAND, gf_budget=0)
    dt = math.comb(12, 7) * ((math.comb(12, 6) + 127) // 128 * 128)
    assert ring >= 4 * 4 * dt * 8  # 4 blocks of p = 4 vectors
    assert full > ring


def test_footprint_rejects_bad_descriptions():
    c = dict(W.plain_2x4())
    c["n_up"] = 9
    with pytest.raises(ed.EDError) as e:
        ed.ed_request_bytes(c)
    assert e.value.status == ed.ED_ERR_INVALID
    c = dict(W.plain_2x4())
    t = np.array(c["t"], dtype=float)
    t[0, 1] += 0.5
    c["t"] = t
    with pytest.raises(ed.EDError):
        ed.ed_request_bytes(c)


def test_band_reserves_ring_unless_all_blocks_fit():
    """A band request reserves every Krylov block only when they all fit the budget; one byte
    less and it reserves its ring of blocks, the only storage it can then use."""
    c = W.cdmft_2x2_bath()
    full = ed.ed_request_bytes(c, n_freq=64, gf_method=ed.ED_GF_BAND, gf_budget=0)
    ring = ed.ed_request_bytes(c, n_freq=64, gf_method=ed.ED_GF_BAND, gf_budget=1)
    # the Green-function part of `full` is the budget at which everything fits
    lo, hi = 1, full
    while hi - lo > 1:  # smallest budget that still reserves the full storage
        mid = (lo + hi) // 2
        if ed.ed_request_bytes(c, n_freq=64, gf_method=ed.ED_GF_BAND, gf_budget=mid) == full:
            hi = mid
        else:
            lo = mid
    assert ed.ed_request_bytes(c, n_freq=64, gf_method=ed.ED_GF_BAND, gf_budget=hi) == full
    assert ed.ed_request_bytes(c, n_freq=64, gf_method=ed.ED_GF_BAND, gf_budget=hi - 1) == ring
    # continued fractions use whatever fits between one run's vectors and all runs'
    cf_lo = ed.ed_request_bytes(c, n_freq=64, gf_budget=1)
    cf_mid = ed.ed_request_bytes(c, n_freq=64, gf_budget=64 << 20)
    cf_hi = ed.ed_request_bytes(c, n_freq=64, gf_budget=0)
    assert cf_lo < cf_mid <= cf_hi
