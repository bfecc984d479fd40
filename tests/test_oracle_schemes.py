"""P12: the oracle's receive-angle schemes against the properties the paper
states for them (Section II-C, Eq. (uniform); Section II-D, Eq. (confocal);
Fig. 2, Fig. 3) and against the compression factors it prints."""
import os

import numpy as np
import pytest

from oracle import schemes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "compression_ratios.txt")


def _tx(N, theta_max_deg=12.0):
    return np.deg2rad(np.linspace(-theta_max_deg, theta_max_deg, N))


def _dtheta_sorted(ps):
    return np.sort(schemes.paraxial_differences(ps))


@pytest.mark.parametrize("N,M", [(15, 15), (7, 7), (15, 57), (11, 5), (75, 129)])
def test_p12a_vernier_is_non_redundant(N, M):
    """j = 0 with odd M: all N*M paraxial differences are distinct ('minimum
    redundancy').  Catches a vernier step that collides with the transmit grid."""
    ps = schemes.scheme("vernier", _tx(N), M)
    d = _dtheta_sorted(ps)
    dth = schemes.transmit_spacing(_tx(N))
    assert d.shape[0] == N * M
    assert np.min(np.diff(d)) > 1e-6 * dth


@pytest.mark.parametrize("N,M", [(15, 15), (7, 7), (15, 57), (11, 5)])
def test_p12b_vernier_support(N, M):
    """Range of Delta theta = (N - 1 + 2 (M-1)/M) dtheta_i, i.e. the transmit
    support widened by about 2/N (Delta k_x = Delta k_ix (1 + 2/N))."""
    tx = _tx(N)
    dth = schemes.transmit_spacing(tx)
    d = _dtheta_sorted(schemes.scheme("vernier", tx, M))
    rng = d[-1] - d[0]
    assert abs(rng - (N - 1 + 2 * (M - 1) / M) * dth) <= 1e-12
    ratio = rng / ((N - 1) * dth)
    # the paper's 1 + 2/N takes Delta k_ix ~ N dk_ix; the exact ratio differs by
    # at most 2/(N(N-1)) + 2/(M(N-1))
    assert abs(ratio - (1 + 2.0 / N)) <= 2.0 / (N * (N - 1)) + 2.0 / (M * (N - 1)) + 1e-12


@pytest.mark.parametrize("N,M", [(15, 15), (7, 7), (15, 57), (11, 5)])
def test_p12c_vernier_step(N, M):
    """Receive angles of one transmit are 2 dtheta_i / M apart, and no gap in
    the sorted differences exceeds that step."""
    tx = _tx(N)
    dth = schemes.transmit_spacing(tx)
    rx = schemes.rx_vernier(dth, M)
    assert np.allclose(np.diff(rx), 2 * dth / M, rtol=0, atol=1e-15)
    d = _dtheta_sorted(schemes.scheme("vernier", tx, M))
    assert np.max(np.diff(d)) <= 2 * dth / M + 1e-12


@pytest.mark.parametrize("N,M", [(15, 15), (7, 7), (15, 57)])
def test_p12d_full_shift_doubles_support(N, M):
    """j = floor(N/2) gives a Delta theta range of about twice the transmit
    range; exact value 2 dtheta_i ((N-1)/2 + (M-1)/M + floor(N/2))."""
    tx = _tx(N)
    dth = schemes.transmit_spacing(tx)
    j = N // 2
    d = _dtheta_sorted(schemes.scheme("shifted", tx, M, j=j))
    rng = d[-1] - d[0]
    assert abs(rng - 2 * dth * ((N - 1) / 2 + (M - 1) / M + j)) <= 1e-12
    assert 1.8 <= rng / ((N - 1) * dth) <= 2.4
    d0 = _dtheta_sorted(schemes.scheme("vernier", tx, M))
    assert rng > 1.6 * (d0[-1] - d0[0])


def test_p12_intermediate_shift_is_bimodal_denser_inside():
    """Intermediate j: denser sampling for |Delta theta| below about
    (N/2 - j) dtheta_i than beyond it."""
    N = M = 15
    tx = _tx(N)
    dth = schemes.transmit_spacing(tx)
    j = 3
    d = schemes.paraxial_differences(schemes.scheme("shifted", tx, M, j=j))
    edge = (N / 2 - j) * dth
    inner = np.sum(np.abs(d) < edge) / (2 * edge)
    outer_w = (d.max() - d.min()) - 2 * edge
    outer = np.sum(np.abs(d) >= edge) / outer_w
    assert inner > 1.3 * outer


def _hist_fit_residuals(d, bins=15):
    h, e = np.histogram(d, bins=bins)
    c = 0.5 * (e[1:] + e[:-1])
    half = max(abs(e[0]), abs(e[-1]))
    tri = 1.0 - np.abs(c) / half
    uni = np.ones_like(c)
    res = []
    for basis in (tri, uni):
        a = np.dot(basis, h) / np.dot(basis, basis)
        res.append(float(np.sum((h - a * basis) ** 2)))
    return res


def test_p12e_confocal_histogram_is_triangular():
    """Eq. (confocal), N = M = 15 over +-12 deg (Fig. 3): a triangle fits the
    Delta theta histogram better than a flat distribution; the vernier (j=0)
    histogram is the other way round."""
    tx = _tx(15)
    d = schemes.paraxial_differences(schemes.scheme("confocal", tx, 15))
    tri, uni = _hist_fit_residuals(d)
    assert tri < 0.5 * uni
    dv = schemes.paraxial_differences(schemes.scheme("shifted", tx, 15, j=7))
    tri_v, uni_v = _hist_fit_residuals(dv)
    assert uni_v < tri_v


def test_confocal_closed_form_entries():
    """Eq. (confocal) for N = 15, M = 15: |o| = 7 gives (14/15 + mod(7, 7)) dtheta
    and |o| = 6 gives (12/15 + 6) dtheta."""
    dth = 1.0
    rx = schemes.rx_confocal(dth, 15, 15)
    assert rx[0] == pytest.approx(-(14 / 15 + 0))
    assert rx[1] == pytest.approx(-(12 / 15 + 6))
    assert rx[7] == 0.0
    assert rx[14] == pytest.approx(14 / 15)


def test_strided_subsets():
    assert list(schemes.strided_subset(75, 8)) == [2, 12, 22, 32, 42, 52, 62, 72]
    assert list(schemes.strided_subset(75, 6)) == [2, 16, 30, 44, 58, 72]
    assert list(schemes.strided_subset(11, 11)) == list(range(11))


def test_golden_compression_factors():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 10
    for r in rows:
        L, N, M, J = (int(v) for v in r[:4])
        printed, decimals = float(r[4]), int(r[5])
        tx = _tx(N)
        if J == 1:
            ps = schemes.scheme("vernier", tx, M)
        else:
            ps = schemes.scheme("hybrid", tx, M, js=[0, 3, 6])
        assert ps.n_groups == J
        assert round(ps.compression_factor(L), decimals) == pytest.approx(printed), r
