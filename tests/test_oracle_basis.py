"""Pins of the oracle's plane-wave basis against closed forms and hand-written
fixtures (CPU only)."""
import os

import numpy as np
import pytest

from oracle import basis as ob

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return np.array([[int(x) for x in r] for r in rows])


@pytest.mark.parametrize("a,ecut_ry,npw,fft", [(10.0, 20.0, 1503, 30), (20.0, 40.0, 34265, 90),
                                               (30.0, 50.0, 161235, 144)])
def test_cubic_counts_and_box(a, ecut_ry, npw, fft):
    """Npw by an integer-only route (m1^2+m2^2+m3^2 <= 2 ecut/b^2) and the box rule
    N >= 4 mmax + 1, even, 2/3/5-smooth."""
    b = ob.sphere(np.diag([a] * 3), [0, 0, 0], ecut_ry / 2)
    bb = 2 * np.pi / a
    lim = (ecut_ry) / bb ** 2          # 2*ecut_ha / b^2
    M = int(np.sqrt(lim)) + 1
    r = np.arange(-M, M + 1)
    n2 = r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2
    assert b.npw == npw == int((n2 <= lim).sum())
    assert b.fft == (fft, fft, fft)
    # Npw follows the sphere volume Omega G_c^3 / (6 pi^2) to a few percent
    est = a ** 3 * (ecut_ry) ** 1.5 / (6 * np.pi ** 2)
    assert abs(b.npw / est - 1) < 0.05


def test_shell_multiplicities_are_sums_of_three_squares():
    fix = _load("free_electron_shells.txt")
    a = 7.0
    bb = 2 * np.pi / a
    b = ob.sphere(np.diag([a] * 3), [0, 0, 0], 0.5 * bb ** 2 * 20.5)
    n = np.rint(b.q2 / bb ** 2).astype(int)
    assert np.allclose(n * bb ** 2, b.q2, rtol=1e-12, atol=0)
    for nn, mult in fix:
        assert (n == nn).sum() == mult


def test_public_order_matches_handwritten_fixture():
    fix = _load("sphere_order_cubic.txt")
    for a in (6.0, 10.0, 13.7):
        b = ob.sphere(np.diag([a] * 3), [0, 0, 0], 4.0 * (2 * np.pi / a) ** 2)
        np.testing.assert_array_equal(b.miller[:19], fix)


def test_order_rules_general_cell():
    lat = np.array([[7.0, 0.3, 0.0], [0.5, 8.0, 0.2], [0.1, -0.4, 9.0]])
    k = np.array([0.25, -0.25, 0.25])
    b = ob.sphere(lat, k, 6.0)
    assert np.all(np.diff(b.q2) >= -1e-10 * b.q2[1:])
    assert np.all(0.5 * b.q2 <= 6.0)
    # inside each shell: strictly lexicographic
    for s in np.unique(b.shell)[:50]:
        m = b.miller[b.shell == s]
        keys = [tuple(x) for x in m]
        assert keys == sorted(keys)
    # every candidate just outside is excluded (completeness): brute force in a bigger box
    r = np.arange(-25, 26)
    M = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    inside = 0.5 * ob.kplusg_sq(lat, k, M) <= 6.0
    assert inside.sum() == b.npw


def test_smooth_sizes():
    assert [ob.smooth_even_at_least(n) for n in (29, 81, 133, 1, 7)] == [30, 90, 144, 2, 8]
