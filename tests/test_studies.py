"""Host-side checks of the flow-study post-processing (no GPU): the Strouhal
estimate recovers the frequency of a synthetic lift signal, with and without
noise and offset, and reports no period for steady or noise-only signals."""
import numpy as np
import pytest

from paper_1601_06984_gb300.studies import _outlet, _strouhal


@pytest.mark.parametrize("period", [569.0, 601.3, 240.0])
def test_strouhal_of_a_sinusoid(period):
    t = np.arange(4000)
    D, U, dt = 40.0, 0.05, 8
    exact = D / (period * dt * U)
    rng = np.random.default_rng(7)
    clean = 0.35 * np.sin(2 * np.pi * t / period + 0.3) + 1.47
    noisy = clean + 0.2 * rng.standard_normal(t.size)
    assert abs(_strouhal(clean, dt, D, U) - exact) < 2e-3 * exact
    assert abs(_strouhal(noisy, dt, D, U) - exact) < 5e-3 * exact


def test_strouhal_none_without_a_period():
    rng = np.random.default_rng(8)
    t = np.arange(4000)
    assert _strouhal(np.zeros(1000), 8, 40.0, 0.05) is None
    assert _strouhal(1e-3 * rng.standard_normal(4000), 8, 40.0, 0.05) is None
    # a steady lift with a decaying wiggle of 1e-4
    assert _strouhal(0.011 + 1e-4 * np.exp(-t / 800) * np.sin(t / 3.0), 8, 40.0, 0.05) is None


def test_outlet_choice():
    assert _outlet("auto", 1.86) == ("linear", 0)
    assert _outlet("auto", 1.97) == ("zero-gradient", 1)
    assert _outlet("linear", 1.97) == ("linear", 0)
