"""The seeded input recipe (the arrays both the oracle and the CUDA path
receive) has the stated properties: contrasts, geometric midrange, forcing
on unknown faces only, mean-free divergence data, inclusion geometry, the
bubble's inside/outside values and the batched size mix."""
import math

import numpy as np
import pytest

from paper_1308_4605_gb300 import workloads as wl


def _ratio(a):
    return float(a.max() / a.min())


@pytest.mark.parametrize("make,rho_c,mu_c", [(lambda: wl.config_c1(32), 10.0, 10.0),
                                             (lambda: wl.config_c3(16), 1e2, 1e3),
                                             (lambda: wl.config_c4_instance(3, 64), 1.0, 1e3),
                                             (lambda: wl.config_c5(16), 1.0, 1e2)])
def test_contrast_and_midrange(make, rho_c, mu_c):
    pr = make()
    for f, c in ((pr.rho, rho_c), (pr.mu, mu_c)):
        assert abs(_ratio(f) - c) <= 1e-9 * c
        assert abs(math.sqrt(float(f.max() * f.min())) - 1.0) <= 1e-12


def test_forcing_on_unknown_faces_and_mean_free_g():
    for pr in (wl.config_c5(16), wl.generic(2, (16, 8), (1, 1, 2, 2, 0, 0), seed=3)):
        for a in range(pr.dim):
            f = pr.b_u[a]
            if pr.bc[2 * a] != wl.PERIODIC:
                sl = [slice(None)] * 3
                sl[2 - a] = 0
                assert not f[tuple(sl)].any()
                sl[2 - a] = -1
                assert not f[tuple(sl)].any()
            assert np.abs(f).max() > 0.5       # N(0,1) on the unknown faces
        assert abs(float(pr.b_p.mean())) <= 1e-12
    assert not wl.config_c5(16).b_p.any()     # the adjoint workload has g = 0
    c3 = wl.config_c3(16)
    assert abs(float(c3.b_p.mean())) <= 1e-12 and float(c3.b_p.std()) > 0.5


def test_inclusions_geometry():
    n = 256
    mu, disks = wl.inclusions_2d((n, n, 1), 1.0, 5)
    assert len(disks) == 20
    L = float(n)
    for i, (cx, cy, r) in enumerate(disks):
        assert 0.02 * L <= r <= 0.06 * L
        assert r <= cx <= L - r and r <= cy <= L - r
        for cx2, cy2, r2 in disks[i + 1:]:
            assert math.hypot(cx - cx2, cy - cy2) > r + r2
    assert set(np.unique(mu)) == {1.0, 1e4}


def test_bubble_values():
    pr = wl.bubble(2, 64, 100.0, 100.0)
    n = 64
    centre = pr.mu[0, n // 2, n // 2]
    corner = pr.mu[0, 0, 0]
    assert 1.0 <= centre <= 1.1 + 1e-12          # inside: 1 + 0.1 U(0, 1), tanh saturated
    assert 100.0 - 1e-9 <= corner <= 100.1 + 1e-12
    assert pr.bc[:4] == (wl.NOSLIP,) * 4 and pr.theta == 0.0


def test_batched_sizes():
    sizes = wl.config_c4_sizes()
    assert len(sizes) == 64 and set(sizes) <= {64, 128, 256, 512}
    assert len(set(sizes)) == 4
