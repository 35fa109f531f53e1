"""Accuracy of the Newton-refined barrier step that the mixed-precision kernels use
(Eqs. Simple-Update:Barrier-X and Simple-Update:Dual, reading A9), restated on the CPU.

The device routine takes the larger root L of t^2 - |omega| t - c = 0 from an FP32
square root of the discriminant, refines it by one Newton step in FP64 (derivative from
the FP32 estimate), and forms the smaller root c / L from an FP32 reciprocal refined by
one Newton step.  FP32 square root and division are IEEE correctly rounded (the compiler's
default), so numpy's float32 operations reproduce the estimates; the device may fuse a
multiply-add where this restatement rounds twice, which the bound covers.  The claim
pinned here: relative error below 2e-14 against the closed form over omega in
+-[1e-12, 1e12] and c in [1e-15, 1e2], and the product x s = c.
"""
import numpy as np


def _closed(omega, c):
    D = np.sqrt(omega * omega + 4.0 * c)
    pos = omega >= 0
    with np.errstate(divide="ignore", invalid="ignore"):   # the branch not taken may divide by 0
        x = np.where(pos, 0.5 * (omega + D), 2.0 * c / (D - omega))
        s = np.where(pos, 2.0 * c / (omega + D), 0.5 * (D - omega))
    return x, s


def _newton(omega, c):
    disc = omega * omega + 4.0 * c
    aw = np.abs(omega)
    d32 = np.sqrt(disc.astype(np.float32))
    L = 0.5 * (aw + d32.astype(np.float64))
    L = L - (L * (L - aw) - c) * (np.float32(1.0) / d32).astype(np.float64)
    r0 = (np.float32(1.0) / L.astype(np.float32)).astype(np.float64)
    small = c * (r0 + r0 * (1.0 - L * r0))
    pos = omega >= 0
    return np.where(pos, L, small), np.where(pos, small, L)


def test_newton_refined_prox_within_2e14_on_its_domain():
    rng = np.random.default_rng(1805)
    n = 400000
    mag = 10.0 ** rng.uniform(-12, 12, n)
    omega = np.where(rng.random(n) < 0.5, -mag, mag)
    c = 10.0 ** rng.uniform(-15, 2, n)
    disc = omega * omega + 4.0 * c
    inside = (disc > 1e-30) & (disc < 1e30)           # the routine's own guard; the rest is closed form
    omega, c = omega[inside], c[inside]
    xr, sr = _closed(omega, c)
    xn, sn = _newton(omega, c)
    ex = np.abs(xn - xr) / xr
    es = np.abs(sn - sr) / sr
    assert inside.mean() > 0.9
    assert ex.max() < 2e-14, ex.max()
    assert es.max() < 2e-14, es.max()
    assert np.max(np.abs(xn * sn - c) / c) < 5e-14


def test_newton_refined_prox_edge_cases():
    """Zero omega (x = s = sqrt(c)), omega far above and below sqrt(c), c at the ends."""
    omega = np.array([0.0, 1e-12, -1e-12, 1e12, -1e12, 3.0, -3.0, 1e-7])
    c = np.array([1e-2, 1e-15, 1e-15, 1e2, 1e2, 1e-15, 1e-15, 1e-14])
    xr, sr = _closed(omega, c)
    xn, sn = _newton(omega, c)
    np.testing.assert_allclose(xn, xr, rtol=2e-14, atol=0)
    np.testing.assert_allclose(sn, sr, rtol=2e-14, atol=0)
    assert np.all(xn > 0) and np.all(sn > 0)
