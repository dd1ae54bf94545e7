"""The element-wise parity check of the GPU tests, on the CPU: an error
confined to one block or one element fails it even where the global relative
L2 over all blocks stays under the bar; rounding-sized errors spread over
every element pass it."""
import numpy as np
import pytest

from parity_checks import K_ELEM, assert_amplitudes_close, parity_report


def _amps(G=64, J=1024, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((G, J)) + 1j * rng.standard_normal((G, J))) / np.sqrt(2 * G * J)


def test_rounding_sized_noise_passes():
    ref = _amps()
    rng = np.random.default_rng(1)
    tol = 1e-5
    # per-element relative noise of RMS 0.8 tol, like an FP32 path at 8e-6
    noise = 0.8 * tol * (rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape)) / np.sqrt(2)
    got = ref + noise * np.sqrt(np.mean(np.abs(ref) ** 2))
    r = assert_amplitudes_close(got, ref, tol)
    assert r["global"] < tol and r["max_block"] < tol


def test_one_wrong_block_is_caught_although_global_passes():
    ref = _amps()
    got = ref.copy()
    got[17] *= 1 + 5e-5  # 5x the bar, in one block of 64
    r = parity_report(got, ref)
    assert r["global"] < 1e-5  # diluted by sqrt(64)
    with pytest.raises(AssertionError, match="worst block"):
        assert_amplitudes_close(got, ref, 1e-5)


def test_one_wrong_element_is_caught_although_blocks_pass():
    ref = _amps()
    got = ref.copy()
    rms = np.sqrt(np.mean(np.abs(ref[3]) ** 2))
    got[3, 100] += 2e-4 * rms  # one element off by 20x the bar's per-element size
    r = parity_report(got, ref)
    assert r["global"] < 1e-5 and r["max_block"] < 1e-5
    assert r["max_elem_over_rms"] > K_ELEM * 1e-5
    with pytest.raises(AssertionError, match="worst element"):
        assert_amplitudes_close(got, ref, 1e-5)


def test_zero_block_must_stay_zero():
    ref = _amps(G=4, J=16)
    ref[2] = 0
    got = ref.copy()
    got[2, 5] = 1e-30
    with pytest.raises(AssertionError, match="zero in the reference"):
        assert_amplitudes_close(got, ref, 1e-5)
