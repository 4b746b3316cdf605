"""Pins of the oracle's correlation, defect, energy-density and Reynolds
observables (Sec. IV) against closed forms, library routines and brute
force, independent of the oracle's own arithmetic."""
import math

import numpy as np
import pytest

from oracle import twofluid as O


def _shell_by_enumeration(nx, ny):
    """Minimum-image shells by explicit loops over displacements."""
    out = np.empty((ny, nx), dtype=np.int64)
    for dy in range(ny):
        for dx in range(nx):
            rx = dx if dx <= (nx - 1) // 2 else dx - nx
            ry = dy if dy <= (ny - 1) // 2 else dy - ny
            out[dy, dx] = int(math.floor(math.sqrt(rx * rx + ry * ry) + 0.5))
    return out


@pytest.mark.parametrize("nx,ny", [(8, 8), (9, 6), (1, 4)])
def test_displacement_shells_by_enumeration(nx, ny):
    shell, n_shell = O.displacement_shells(nx, ny)
    assert np.array_equal(shell, _shell_by_enumeration(nx, ny))
    assert n_shell == min(nx, ny) // 2 + 1


def test_autocorrelation_equals_wiener_khinchin():
    """Direct shifted sums against the library FFT route (Wiener-Khinchin)."""
    rng = np.random.default_rng(4)
    a = rng.standard_normal((2, 6, 10))
    R = O.autocorrelation(a)
    F = np.fft.fft2(a)
    Rw = np.real(np.fft.ifft2((np.abs(F) ** 2).sum(axis=0))) / a[0].size
    assert np.allclose(R, Rw, atol=1e-12)
    # a shift by one site in x pairs a(x) with a(x + 1): check one entry by hand
    want = np.mean((a * np.roll(a, -1, axis=2)).sum(axis=0))
    assert R[0, 1] == pytest.approx(want, abs=1e-14)


@pytest.mark.parametrize("m", [1, 3])
def test_spatial_correlation_of_one_mode(m):
    """a = cos(2 pi m x / nx) has C(r) = cos(2 pi m r_x / nx); the shell
    average is the mean of that over the shell's displacements."""
    nx, ny = 16, 12
    x = np.arange(nx)
    a = np.cos(2 * np.pi * m * x / nx)[None, None, :].repeat(ny, axis=1)
    C = O.spatial_correlation(a, centred=False)
    shell = _shell_by_enumeration(nx, ny)
    n_shell = min(nx, ny) // 2 + 1
    for s in range(n_shell):
        vals = [math.cos(2 * math.pi * m * (dx if dx <= (nx - 1) // 2 else dx - nx) / nx)
                for dy in range(ny) for dx in range(nx) if shell[dy, dx] == s]
        assert C[s] == pytest.approx(np.mean(vals), abs=1e-12)
    assert C[0] == pytest.approx(1.0)


def test_spatial_correlation_centring():
    """A constant offset is removed by centring and kept otherwise."""
    rng = np.random.default_rng(5)
    a = rng.standard_normal((1, 8, 8))
    assert np.allclose(O.spatial_correlation(a + 3.0, True), O.spatial_correlation(a, True))
    C = O.spatial_correlation(np.full((1, 8, 8), 2.0), False)
    assert np.allclose(C, 1.0)


def _state(p, seed=0):
    rng = np.random.default_rng(seed)
    n = (p.ny, p.nx)
    phi = 0.5 + 0.02 * rng.standard_normal(n)
    th = np.pi * rng.random(n)
    s = O.state_from_fields(phi, 0.2 * np.cos(2 * th), 0.2 * np.sin(2 * th), p,
                            u1=0.01 * rng.standard_normal((2,) + n),
                            u2=0.01 * rng.standard_normal((2,) + n))
    return s


def test_time_correlations_identities():
    p = O.Params(nx=12, ny=10)
    s = _state(p)
    assert np.allclose(O.time_correlations(s, s, p), [1.0, 1.0, 1.0])
    flipped = O.State(s.f1, s.f2, s.phi, -s.Qxx, -s.Qxy)
    assert O.time_correlations(s, flipped, p)[2] == pytest.approx(-1.0)


def _director_pair(nx, ny, plus, minus):
    """theta = 1/2 atan2 around `plus` minus 1/2 atan2 around `minus`."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    th = 0.5 * np.arctan2(y - plus[1], x - plus[0]) - 0.5 * np.arctan2(y - minus[1], x - minus[0])
    return np.cos(2 * th), np.sin(2 * th)


def test_defects_of_a_constructed_pair():
    """A +1/2 and a -1/2 defect centred in two plaquettes are found there,
    with the right signs; a uniform director has none."""
    qxx, qxy = _director_pair(32, 32, (10.5, 16.5), (21.5, 16.5))
    q = O.defect_charges(qxx, qxy)
    assert q[16, 10] == 0.5 and q[16, 21] == -0.5
    assert np.count_nonzero(q) == 2
    assert list(O.defect_counts(qxx, qxy)) == [1, 1, 0]
    assert list(O.defect_counts(np.full((8, 8), 0.3), np.full((8, 8), -0.1))) == [0, 0, 0]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_defect_charges_sum_to_zero_on_the_torus(seed):
    """On a periodic grid every edge is walked once in each direction by the
    two plaquettes it borders, so the charges of any director field sum to
    zero; on a four-edge loop a charge is -1/2, 0 or +1/2."""
    rng = np.random.default_rng(seed)
    th = np.pi * rng.random((24, 20))
    q = O.defect_charges(np.cos(2 * th), np.sin(2 * th))
    assert set(np.unique(q)) <= {-0.5, 0.0, 0.5}
    assert q.sum() == 0.0
    assert np.count_nonzero(q) > 0
    n = O.defect_counts(np.cos(2 * th), np.sin(2 * th))
    assert n[0] == n[1] and n[2] == 0


def test_elastic_energy_of_one_mode():
    """Q_xx = S cos(k x), Q_xy = 0: central differences give
    d_x Q_xx = -S sin(k x) sin(k), and Q_yy = -Q_xx doubles the sum, so
    E = K S^2 sin(k)^2 sin(k x)^2."""
    nx, ny, S, K = 16, 4, 0.3, 0.04
    k = 2 * np.pi * 3 / nx
    x = np.arange(nx)
    qxx = (S * np.cos(k * x))[None, :].repeat(ny, axis=0)
    E = O.elastic_energy_density(qxx, np.zeros_like(qxx), K)
    want = (K * S * S * np.sin(k) ** 2 * np.sin(k * x) ** 2)[None, :].repeat(ny, axis=0)
    assert np.allclose(E, want, atol=1e-15)


def test_uniform_flow_energy_and_reynolds():
    """u1 = u2 = U everywhere, uniform phi, Q = 0: no forces, so u_c = U;
    E_kin = (rho1 + rho2) |U|^2 / 2 and Re = (rho1 + rho2) |U| sqrt(K/zeta) /
    (eta1 + eta2) with eta_k = rho_k (tau_k - 1/2)/3."""
    p = O.Params(nx=6, ny=5, rho1=1.1, rho2=0.9, tau1=1.0, tau2=0.8, zeta=0.004, K=0.05)
    U = np.array([0.02, -0.01])
    u = np.broadcast_to(U[:, None, None], (2, 5, 6)).copy()
    z = np.zeros((5, 6))
    s = O.state_from_fields(np.full((5, 6), 0.5), z, z, p, u1=u, u2=u)
    assert np.allclose(O.kinetic_energy_density(s, p), 0.5 * 2.0 * (U @ U), atol=1e-15)
    Re, La = O.reynolds(s, p)
    eta = 1.1 * 0.5 / 3 + 0.9 * 0.3 / 3
    assert La == pytest.approx(math.sqrt(0.05 / 0.004))
    assert Re == pytest.approx(2.0 * math.sqrt(U @ U) * La / eta, rel=1e-12)
