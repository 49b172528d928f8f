"""Validation cases of the paper run through the CUDA path: the sessile-droplet contact angle
of the two-component Shan-Chen model with adhesion (contact-angle section of Sec. 3.2).

The angle is measured as the paper does: the droplet height h and contact length b give the
cap radius r = (4h^2 + b^2) / (8h) and theta = pi - arctan(b / (2(h - r))), the arctangent
taken in the quadrant of (b, 2(h - r)) so that caps lower than a half disc (h < r) give angles
below 90 degrees."""
import numpy as np
import pytest

from paper_2502_12955_gb300 import inputs
from paper_2502_12955_gb300.lbm import Solver

pytestmark = pytest.mark.gpu


def contact_angle(r0):
    """Angle (degrees) of the droplet of component 0 on the wall at y = -1/2.  The interface is
    the mid-density contour; h is its height on the droplet's centre column, b its width on the
    first fluid row, both by linear interpolation between nodes."""
    ny, nx = r0.shape
    hi, lo = float(r0.max()), float(r0.min())
    thr = 0.5 * (hi + lo)
    w = (r0 - lo).clip(0)
    xc = int(round(float((w.sum(axis=0) * np.arange(nx)).sum() / w.sum())))
    col = r0[:, xc]
    yt = int(np.nonzero(col > thr)[0].max())
    h = yt + (col[yt] - thr) / (col[yt] - col[yt + 1]) + 0.5
    row = r0[0]
    inr = np.nonzero(row > thr)[0]
    assert 0 < inr.min() and inr.max() < nx - 1, "the droplet left the wall or wet it entirely"
    xl, xr = int(inr.min()), int(inr.max())
    b = (xr + (row[xr] - thr) / (row[xr] - row[xr + 1])) - (xl - (row[xl] - thr) / (row[xl] - row[xl - 1]))
    r = (4.0 * h * h + b * b) / (8.0 * h)
    return float(np.degrees(np.pi - np.arctan2(b, 2.0 * (h - r)))), hi, lo


def _run(g, steps=60000):
    cfg, geom, fields = inputs.sessile_droplet_2d(g_ads=g)
    s = Solver(cfg)
    s.set_geometry(geom)
    s.set_fields(*fields)
    s.step(steps)
    theta, hi, lo = contact_angle(s.fields()["rho"][0, 0])
    s.close()
    return theta, hi, lo, cfg["G"][0][1]


def test_contact_angle_of_sessile_droplet():
    """Neutral walls give 90 degrees; a wall that repels the droplet's component and attracts the
    other (G_ads = (g, -g), g > 0) gives a non-wetting cap, the opposite sign a wetting one; and
    exchanging the roles of the two components (g -> -g) gives the supplementary angle.  The
    angles are printed beside Huang's closed form cos(theta) = (G_ads,2 - G_ads,1) / (G_c
    (rho_1 - rho_2) / 2) quoted in the paper; the measured cos(theta) has its sign and is larger
    by a factor of 1.7-1.9 at these parameters (65.2 / 90.6 / 117.1 degrees against 75.5 / 90 /
    104.3 on a GB300)."""
    res = {g: _run(g) for g in (-0.15, 0.0, 0.15)}
    for g, (theta, hi, lo, G) in res.items():
        huang = np.degrees(np.arccos(np.clip(-2.0 * g / (G * (hi - lo) / 2.0), -1.0, 1.0)))
        print(f"G_ads = ({g}, {-g}): theta {theta:.2f} deg, Huang {huang:.2f} deg, "
              f"rho {hi:.4f} / {lo:.4f}")
    t_neg, t_0, t_pos = res[-0.15][0], res[0.0][0], res[0.15][0]
    assert abs(t_0 - 90.0) < 2.0
    assert t_pos > 100.0 and t_neg < 80.0
    assert abs((t_pos + t_neg) - 180.0) < 4.0
    # same sign as the closed form, and cos(theta) of the same order
    for g in (-0.15, 0.15):
        theta, hi, lo, G = res[g]
        c_h = -2.0 * g / (G * (hi - lo) / 2.0)
        ratio = np.cos(np.radians(theta)) / c_h
        assert 0.5 < ratio < 3.0, ratio
