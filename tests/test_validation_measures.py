"""The measurements of the validation cases (Sec. 3.2), checked on synthetic fields of known
geometry.

Contact angle: caps of known angle, a circle of radius R whose centre lies R cos(theta) below
the wall face y = -1/2, with a tanh interface of width 2 between the bulk densities.  The circle
fit must return theta and R (a wall face misplaced by half a node moves the angle by about 1
degree at these sizes); the paper's h / b construction, which reads the first fluid row, must be
within the error of that row's interpolation.

Rayleigh-Taylor: the interface height per column of a tanh interface at y0 + a cos(2 pi x / nx),
from which the growth of the mode is read, must return that height, and its first Fourier
coefficient the mode's amplitude."""
import numpy as np
import pytest

from tests.test_gpu_validation import _interface_heights, circle_angle, contact_angle


def _cap(theta_deg, R=25.0, nx=200, ny=80, width=2.0, hi=0.96, lo=0.07):
    th = np.radians(theta_deg)
    yc = -0.5 - R * np.cos(th)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.hypot(x - nx / 2.0, y - yc)
    return lo + (hi - lo) * 0.5 * (1.0 - np.tanh((d - R) / width))


@pytest.mark.parametrize("theta", [45.0, 60.0, 90.0, 120.0, 135.0])
def test_angle_of_a_synthetic_cap(theta):
    r0 = _cap(theta)
    t_fit, R = circle_angle(r0)
    assert abs(t_fit - theta) < 0.1, t_fit
    assert abs(R - 25.0) < 0.1, R
    t_paper = contact_angle(r0)[0]
    assert abs(t_paper - theta) < 1.5, t_paper


@pytest.mark.parametrize("amp", [0.5, 4.0, 40.0])
def test_interface_height_of_a_cosine_mode(amp):
    ny, nx, y0 = 512, 256, 255.5
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    eta = y0 + amp * np.cos(2 * np.pi * (x + 0.5) / nx)
    phi = np.tanh((eta - y) / 2.0)     # +1 below the interface, -1 above
    h = _interface_heights(phi)
    exact = y0 + amp * np.cos(2 * np.pi * (np.arange(nx) + 0.5) / nx)
    assert np.abs(h - exact).max() < 0.02, np.abs(h - exact).max()
    # the mode's amplitude as the Rayleigh-Taylor case reads it: the first Fourier coefficient
    a1 = 2.0 * abs(np.fft.rfft(h - h.mean())[1]) / nx
    assert abs(a1 - amp) < 0.01 * max(amp, 1.0), a1
