"""Host-side checks of the flow-study post-processing (no GPU): the Strouhal
estimate recovers the frequency of a synthetic lift signal, with and without
noise and offset, and reports no period for steady or noise-only signals; the
recirculation length recovers the zero of a synthetic axial velocity on a
three-level mesh."""
import numpy as np
import pytest

from paper_1601_06984_gb300 import workloads as W
from paper_1601_06984_gb300.studies import _outlet, _strouhal, recirculation_length


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


def _axis_field(mesh, fn):
    """u [n, 3] with u_x = fn(x) at the element centres (finest-cell units)."""
    lv = mesh.levels.astype(np.int64)
    h = np.ldexp(1.0, int(lv.max()) - lv)
    x = (mesh.coords[:, 0] + 0.5) * h
    u = np.zeros((mesh.n, 3))
    u[:, 0] = fn(x)
    return u


def test_recirculation_length_of_a_synthetic_wake():
    """Sphere of diameter 8 finest cells at (44, 24, 24) on the three-level
    mesh: an axial velocity that is linear in x (so the interpolation is exact)
    and vanishes 7 cells behind the rear point gives L_r / D = 7/8; a profile
    with its zero between two cell centres, and one with unequal values off
    the axis (only the four cells around the axis count), too."""
    m = W.config_sphere_small()
    c, D = (44.0, 24.0, 24.0), 8.0
    rear = c[0] + D / 2
    u = _axis_field(m, lambda x: 0.01 * (x - (rear + 7.0)))
    assert abs(recirculation_length(m, u, c, D) - 7.0 / 8.0) < 1e-12
    u = _axis_field(m, lambda x: 0.01 * (x - (rear + 6.3)))
    assert abs(recirculation_length(m, u, c, D) - 6.3 / 8.0) < 1e-12
    lv = m.levels.astype(np.int64)
    h = np.ldexp(1.0, int(lv.max()) - lv)
    y = (m.coords[:, 1] + 0.5) * h
    u[np.abs(y - c[1]) > h, 0] = 5.0  # far from the axis: ignored
    assert abs(recirculation_length(m, u, c, D) - 6.3 / 8.0) < 1e-12


def test_recirculation_length_none_without_reversed_flow():
    m = W.config_sphere_small()
    u = _axis_field(m, lambda x: 0.04 + 0.0 * x)
    assert recirculation_length(m, u, (44.0, 24.0, 24.0), 8.0) is None
    u = _axis_field(m, lambda x: -0.01 + 0.0 * x)
    assert recirculation_length(m, u, (44.0, 24.0, 24.0), 8.0) is None
