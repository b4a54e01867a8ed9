"""Host entry points of the detection products in the C ABI that need no
GPU: the paper's additional spectra against the oracle, eq. Threshold from
sums, the refusal of libraries holding the paper's extras, and argument
checks."""
import ctypes

import numpy as np

import oracle.detection as od
import synth
from paper_1402_2518_gb300 import linmin

from .test_oracle_detection import HAND_EXTRAS

def _sums_struct(d):
    s = linmin.linmin_threshold_sums()
    for k, v in d.items():
        arr = getattr(s, k)
        for i, val in enumerate(v):
            arr[i] = val
    return s


def test_c_thresholds_match_oracle():
    """eq. Threshold in the library (host code) from oracle sums equals the
    oracle's two-pass formula."""
    rng = np.random.Generator(np.random.PCG64(8))
    x = rng.uniform(0, 0.1, (5000, 6)).astype(np.float32)
    truth = rng.integers(0, 64, 5000).astype(np.uint64)
    sums = od.threshold_sums(x, truth, 6)
    c = linmin.linmin_thresholds(_sums_struct(sums), 6)
    np.testing.assert_allclose(c, od.thresholds(x, truth, 6).astype(np.float32), rtol=1e-6)
    hand = _sums_struct(od.threshold_sums(np.array([[0.04], [0.06], [0.0], [0.002]], np.float32),
                                          np.array([1, 1, 0, 0], np.uint64), 1))
    assert abs(linmin.linmin_thresholds(hand, 1)[0] - 0.0185) < 1e-8
    empty = _sums_struct({"n_pos": [0], "n_neg": [3]})
    assert np.isnan(linmin.linmin_thresholds(empty, 1)[0])


def test_c_extra_spectra_match_oracle():
    for L, w in ((3, None), (184, None), (240, synth.wavelengths(240).astype(np.float32)),
                 (17, np.sort(np.random.default_rng(1).uniform(1, 2.5, 17)).astype(np.float32))):
        got = linmin.linmin_extra_spectra(L, 12, w)
        want = od.paper_extra_spectra(L, w, 12).astype(np.float32)
        ulp = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
        assert (np.abs(got - want) <= 1e-7).all() or ulp.max() <= 1, (L, ulp.max())
    np.testing.assert_allclose(linmin.linmin_extra_spectra(3, 4), HAND_EXTRAS[:4], atol=1e-7)


def test_create_refuses_paper_extras():
    rng = np.random.Generator(np.random.PCG64(4))
    mins = synth.library(rng, 184, 32, 0).astype(np.float32)
    for n in (4, 12):
        S = np.ascontiguousarray(np.vstack([mins, linmin.linmin_extra_spectra(184, n)]))
        h = ctypes.c_void_p()
        st = linmin.lib().linmin_create(S.ctypes.data_as(ctypes.c_void_p), 184, S.shape[0], None,
                                        ctypes.byref(h))
        assert st == linmin.LINMIN_ERR_RANK


def test_detection_arguments_rejected_on_host():
    lib = linmin.lib()
    xm = np.zeros(4, np.float32)
    P_ = ctypes.c_void_p
    xmp = xm.ctypes.data_as(P_)
    inv = linmin.LINMIN_ERR_INVALID
    assert lib.linmin_detect(None, None, None, None, None, 10, 0, 0, xmp, 1.0, None, None, None) == inv
    assert lib.linmin_detect(None, None, None, None, None, 10, 65, 0, xmp, 1.0, None, None, None) == inv
    assert lib.linmin_detect(None, None, None, None, None, 10, 4, 5, xmp, 1.0, None, None, None) == inv
    assert lib.linmin_detect(None, None, None, None, None, -1, 4, 4, xmp, 1.0, None, None, None) == inv
    assert lib.linmin_detect(None, None, None, None, None, 10, 4, 4, xmp, 1.0, None, None, None) == inv
    xm[1] = -0.1
    assert lib.linmin_detect(None, None, None, None, None, 0, 4, 4, xmp, 1.0, None, None, None) == inv
    assert "x_min" in linmin.linmin_last_error(None)
    assert lib.linmin_threshold_stats(None, None, 10, 4, 4, None, None) == inv
    assert lib.linmin_extra_spectra(1, None, 12, xmp) == inv
    assert lib.linmin_extra_spectra(8, None, 5, xmp) == inv
    w = np.array([1.0, 0.5, 2.0], np.float32)
    out = np.empty((12, 3), np.float32)
    assert lib.linmin_extra_spectra(3, w.ctypes.data_as(P_), 12, out.ctypes.data_as(P_)) == inv


def test_second_pass_and_autofit_arguments_rejected_on_host():
    lib = linmin.lib()
    P_ = ctypes.c_void_p
    S = np.ones((4, 16), np.float32)
    sp = S.ctypes.data_as(P_)
    inv = linmin.LINMIN_ERR_INVALID
    # n_minerals must leave at least one always-kept column
    assert lib.linmin_second_pass(sp, 16, 4, 4, None, None, 0, None, None, None, None, None,
                                  None) == inv
    assert lib.linmin_second_pass(sp, 16, 0, 0, None, None, 0, None, None, None, None, None,
                                  None) == inv
    assert lib.linmin_second_pass(None, 16, 4, 2, None, None, 0, None, None, None, None, None,
                                  None) == inv
    assert lib.linmin_unmix_masked(None, None, 0, None, None, 0, None, None, None, None) == inv
    assert lib.linmin_autofit(sp, 16, 1, None, None, None, None, None, None, None) == inv
    assert lib.linmin_autofit(sp, 3, 4, None, None, None, None, None, None, None) == inv
    assert lib.linmin_autofit(None, 16, 4, None, None, None, None, None, None, None) == inv
