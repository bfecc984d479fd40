"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names the mistake it is there to catch.  All run on CPU.
"""
from fractions import Fraction

import numpy as np
import pytest

import kksynth
from oracle import kk, schemes
from tests import bruteforce

FS, C = kksynth.FS, kksynth.C_SOUND


# ----------------------------------------------------------------------------
# P1: brute force on tiny inputs (vectorisation mistakes: axes, transposes)
# ----------------------------------------------------------------------------
def test_p1_bruteforce_kk_and_das():
    w = kksynth.workload_tiny(seed=3, n_elem=4, n_tx=2, n_samples=32, nx=8, nz=8)
    ps = schemes.full_product(w.tx_angles, [0, 1],
                              [np.deg2rad([-5.0, 0.0, 7.0]), np.deg2rad([3.0])])
    B = kk.kk_image(w.rf, w.elem_x, ps, w.grid, w.fs, w.c)
    px, pz = kk.grid_pixels(w.grid)
    pairs = [(int(i), float(ps.rx_angles[o])) for i, o in zip(ps.tx_index, ps.rx_index)]
    rf = w.rf.astype(np.float64).tolist()
    ref = bruteforce.kk_chain(rf, list(w.elem_x), list(w.tx_angles), pairs,
                              [int(g) for g in ps.group], ps.n_groups,
                              list(zip(px, pz)), w.fs, w.c)
    ref = np.array(ref).reshape(B.shape)
    assert np.abs(ref).max() > 0
    assert kk.rel_l2(B, ref) <= 1e-12
    D = kk.das_image(w.rf, w.tx_angles, w.elem_x, w.grid, w.fs, w.c)
    refd = np.array(bruteforce.das_chain(rf, list(w.elem_x), list(w.tx_angles),
                                         list(zip(px, pz)), w.fs, w.c)).reshape(D.shape)
    assert kk.rel_l2(D, refd) <= 1e-12


# ----------------------------------------------------------------------------
# P8: analytic signal (dropped factor 2, wrong 1/T, Nyquist handling)
# ----------------------------------------------------------------------------
def test_p8_analytic_real_part_is_rf_minus_nyquist():
    rng = np.random.default_rng(0)
    T = 64
    rf = rng.standard_normal((3, T))
    y = kk.analytic_signal(rf)
    t = np.arange(T)
    nyq = (rf * (-1.0) ** t).sum(axis=-1, keepdims=True) / T * (-1.0) ** t
    assert np.abs(y.real - (rf - nyq)).max() <= 1e-12


@pytest.mark.parametrize("k0,phi", [(1, 0.3), (5, -1.1), (31, 2.0)])
def test_p8_analytic_of_a_tone_is_the_complex_exponential(k0, phi):
    T = 64
    t = np.arange(T)
    rf = 1.7 * np.cos(2 * np.pi * k0 * t / T + phi)
    y = kk.analytic_signal(rf)
    assert np.abs(y - 1.7 * np.exp(1j * (2 * np.pi * k0 * t / T + phi))).max() <= 1e-12


def test_p8_analytic_of_dc_is_dc():
    y = kk.analytic_signal(np.full(16, 2.5))
    assert np.abs(y - 2.5).max() <= 1e-13


# ----------------------------------------------------------------------------
# P2: Fourier-shift shear equals a time-domain circular advance when every
# shift is a whole number of samples (sign of the phase, x_ref rule, fs/T)
# ----------------------------------------------------------------------------
def test_p2_fourier_shear_is_integer_time_advance():
    pitch = 0.3e-3
    L, T = 9, 128
    s1 = C / (FS * pitch)          # pitch * sin(theta) * fs / c == 1
    th = np.arcsin(s1)
    w = kksynth.workload_custom("p2", 5, L, pitch, 3, 8.0, T, (4, 4, -1e-3, 0.5e-3, 3e-3, 0.5e-3),
                                kksynth.point_phantom([(0.5, 3.0), (-0.7, 4.0)]), snr_db=20.0)
    rx = np.array([-th, 0.0, th])
    ps = schemes.full_product(w.tx_angles, [0, 1, 2], [rx])
    y = kk.decompose(w.rf, w.elem_x, ps, FS, C)
    a = kk.analytic_signal(w.rf)                   # [N][L][T]
    for p in range(ps.n_pairs):
        i, o = ps.tx_index[p], ps.rx_index[p]
        # advance of element l, in samples, when the shear reference is the
        # far array end for the sign of theta: (L-1-l) for theta > 0, l for < 0
        if rx[o] > 0:
            shifts = [L - 1 - l for l in range(L)]
        elif rx[o] < 0:
            shifts = list(range(L))
        else:
            shifts = [0] * L
        ref = sum(np.roll(a[i, l], -shifts[l]) for l in range(L))
        assert np.abs(y[p] - ref).max() <= 1e-11 * np.abs(ref).max()


# ----------------------------------------------------------------------------
# P6: KK image formation on synthetic records with integral delays, worked by
# hand (transposed sin/cos, wrong x_ref, off-by-one sample, lerp weights,
# record-end rule).
#
# Geometry in units of q = c / fs: transmit and receive angles in
# {-a, 0, +a} with sin a = 0.28, cos a = 0.96; 11 elements at pitch 5q, so
# the array ends are at +-25q (x_ref = 25q for +a, -25q for -a).
# For pixel (x, z) and pair (i, o) the KK sample position is
#   s = x sin_i + z cos_i + (x - x_ref) sin_o + z cos_o       (in samples).
# At the lattice pixels below every s is an integer (25 * 0.28 = 7,
# 25 * 0.96 = 24), tabulated by hand in EXPECTED_S.
# ----------------------------------------------------------------------------
Q = C / FS
SIN_A, COS_A = 0.28, 0.96


def _p6_geometry():
    a = np.arcsin(SIN_A)
    angles = np.array([-a, 0.0, a])
    elem_x = (np.arange(11) - 5.0) * 5 * Q
    ps = schemes.full_product(angles, [0, 1, 2], [angles])
    return angles, elem_x, ps


# pixel (x/q, z/q) -> s for pairs ordered (i, o) over {-a, 0, +a}^2
def _s_by_hand(xq, zq):
    sc = {-1: (Fraction(-28, 100), Fraction(96, 100)), 0: (Fraction(0), Fraction(1)),
          1: (Fraction(28, 100), Fraction(96, 100))}
    xref = {-1: -25, 0: 0, 1: 25}
    out = []
    for i in (-1, 0, 1):
        for o in (-1, 0, 1):
            si, ci = sc[i]
            so, co = sc[o]
            out.append(xq * si + zq * ci + (xq - xref[o]) * so + zq * co)
    return out


EXPECTED_S = {
    (0, 25): [41, 49, 41, 42, 50, 42, 41, 49, 41],
    (25, 50): [75, 91, 89, 84, 100, 98, 89, 105, 103],
    (-25, 50): [103, 105, 89, 98, 100, 84, 89, 91, 75],
}


def test_p6_hand_table_is_consistent():
    for (xq, zq), s in EXPECTED_S.items():
        assert [int(v) for v in _s_by_hand(xq, zq)] == s
        assert all(v.denominator == 1 for v in _s_by_hand(xq, zq))


def test_p6_kk_integral_delays_pick_exact_samples():
    angles, elem_x, ps = _p6_geometry()
    T = 160
    rng = np.random.default_rng(11)
    y = rng.standard_normal((ps.n_pairs, T)) + 1j * rng.standard_normal((ps.n_pairs, T))
    pix = list(EXPECTED_S.keys())
    grid = (1, 1, 0.0, Q, 0.0, Q)   # x = ix * q, z = iz * q
    B = kk.kk_beamform(y, elem_x, ps, grid, FS, C, pixels=[(x, z) for x, z in pix])[0]
    for q_, key in enumerate(pix):
        ref = sum(y[p, EXPECTED_S[key][p]] for p in range(ps.n_pairs))
        assert abs(B[q_] - ref) <= 1e-12 * abs(ref)


def test_p6_lerp_weights_and_record_end_on_linear_records():
    """Records linear in t make linear interpolation exact: the image at a
    quarter-sample offset is sum_p (a_p + b_p s_p) over pairs whose k = floor(s)
    keeps k+1 inside the record, 0 for the others."""
    angles, elem_x, ps = _p6_geometry()
    rng = np.random.default_rng(12)
    a = rng.standard_normal(ps.n_pairs) + 1j * rng.standard_normal(ps.n_pairs)
    b = rng.standard_normal(ps.n_pairs) + 1j * rng.standard_normal(ps.n_pairs)
    # pixel (0, 25q + q/4): s = s(0,25) + (cos_i + cos_o)/4, i.e. +0.48, +0.49 or +0.5
    cos_of = {-1: Fraction(96, 100), 0: Fraction(1), 1: Fraction(96, 100)}
    order = [(i, o) for i in (-1, 0, 1) for o in (-1, 0, 1)]
    s_exact = [EXPECTED_S[(0, 25)][p] + (cos_of[i] + cos_of[o]) / 4
               for p, (i, o) in enumerate(order)]
    for T in (43, 44, 60):
        t = np.arange(T)
        y = a[:, None] + b[:, None] * t[None, :]
        grid = (1, 1, 0.0, Q, 25 * Q + Q / 4, Q)
        B = kk.kk_beamform(y, elem_x, ps, grid, FS, C, pixels=[(0, 0)])[0, 0]
        ref = 0j
        for p in range(ps.n_pairs):
            s = float(s_exact[p])
            k = int(np.floor(s))
            if k >= 0 and k + 1 <= T - 1:
                ref += a[p] + b[p] * s
        assert abs(B - ref) <= 1e-11 * max(abs(ref), 1.0), T


# ----------------------------------------------------------------------------
# P13: DAS with integral delays (3-4-5 geometry): the sum picks y_il at the
# hand-computed sample of every (transmit, element).
#   q = c/fs, pixel (0, 40q), elements at {-30, 0, 30} q, transmit angles with
#   cos in {0.75, 1, 0.75}:  tau_in = 40 cos_i -> {30, 40, 30},
#   tau_out = {50, 40, 50}  =>  s_il = tau_in + tau_out.
# ----------------------------------------------------------------------------
def test_p13_das_integral_delays():
    b = np.arccos(0.75)
    tx = np.array([-b, 0.0, b])
    elem_x = np.array([-30.0, 0.0, 30.0]) * Q
    s_hand = [[80, 70, 80], [90, 80, 90], [80, 70, 80]]
    T = 100
    rng = np.random.default_rng(5)
    y = rng.standard_normal((3, 3, T)) + 1j * rng.standard_normal((3, 3, T))
    B = kk.das_beamform_analytic(y, tx, elem_x, (1, 1, 0.0, Q, 40 * Q, Q), FS, C)[0, 0]
    ref = sum(y[i, l, s_hand[i][l]] for i in range(3) for l in range(3))
    assert abs(B - ref) <= 1e-12 * abs(ref)
    # a unit spike at each hand-computed sample gives N * L
    y2 = np.zeros_like(y)
    for i in range(3):
        for l in range(3):
            y2[i, l, s_hand[i][l]] = 1.0
    B2 = kk.das_beamform_analytic(y2, tx, elem_x, (1, 1, 0.0, Q, 40 * Q, Q), FS, C)[0, 0]
    assert abs(B2 - 9.0) <= 1e-12


# ----------------------------------------------------------------------------
# P3: linearity; P11: additivity over pairs and groups
# ----------------------------------------------------------------------------
def test_p3_linearity_kk_and_das():
    wa = kksynth.workload_tiny(seed=21, n_elem=6, n_tx=3, n_samples=64, nx=10, nz=9)
    wb = kksynth.workload_tiny(seed=22, n_elem=6, n_tx=3, n_samples=64, nx=10, nz=9)
    ps = schemes.scheme("vernier", wa.tx_angles, 5)
    al, be = 0.7, -2.3
    mix = (al * wa.rf.astype(np.float64) + be * wb.rf.astype(np.float64))
    Ba = kk.kk_image(wa.rf, wa.elem_x, ps, wa.grid, FS, C)
    Bb = kk.kk_image(wb.rf, wa.elem_x, ps, wa.grid, FS, C)
    Bm = kk.kk_image(mix, wa.elem_x, ps, wa.grid, FS, C)
    assert kk.rel_l2(Bm, al * Ba + be * Bb) <= 1e-12
    Da = kk.das_image(wa.rf, wa.tx_angles, wa.elem_x, wa.grid, FS, C)
    Db = kk.das_image(wb.rf, wa.tx_angles, wa.elem_x, wa.grid, FS, C)
    Dm = kk.das_image(mix, wa.tx_angles, wa.elem_x, wa.grid, FS, C)
    assert kk.rel_l2(Dm, al * Da + be * Db) <= 1e-12


def test_p11_additivity_over_pairs_and_groups():
    w = kksynth.workload_tiny(seed=23, n_elem=6, n_tx=3, n_samples=64, nx=7, nz=6)
    dth = schemes.transmit_spacing(w.tx_angles)
    r1, r2 = schemes.rx_shifted(dth, 3, 0), schemes.rx_shifted(dth, 3, 1)
    g1 = schemes.full_product(w.tx_angles, [0, 1, 2], [r1])
    g2 = schemes.full_product(w.tx_angles, [0, 1, 2], [r2])
    both = schemes.full_product(w.tx_angles, [0, 1, 2], [r1, r2])
    one = schemes.PairSet(both.tx_angles, both.rx_angles, both.tx_index, both.rx_index,
                          np.zeros_like(both.group), 1)
    B1 = kk.kk_image(w.rf, w.elem_x, g1, w.grid, FS, C)[0]
    B2 = kk.kk_image(w.rf, w.elem_x, g2, w.grid, FS, C)[0]
    Bboth = kk.kk_image(w.rf, w.elem_x, both, w.grid, FS, C)
    Bone = kk.kk_image(w.rf, w.elem_x, one, w.grid, FS, C)[0]
    assert kk.rel_l2(Bboth[0], B1) <= 1e-13 and kk.rel_l2(Bboth[1], B2) <= 1e-13
    assert kk.rel_l2(Bone, B1 + B2) <= 1e-12
    I_coh = kk.compound(Bboth, "coherent")
    I_inc = kk.compound(Bboth, "incoherent")
    assert np.allclose(I_coh, np.abs(B1 + B2) ** 2, rtol=1e-12, atol=0)
    assert np.allclose(I_inc, np.abs(B1) ** 2 + np.abs(B2) ** 2, rtol=1e-12, atol=0)


# ----------------------------------------------------------------------------
# P9: x_ref invariance (the shear reference only moves the record's time
# origin; a wrong pairing between the shear and tau_out breaks this)
# ----------------------------------------------------------------------------
def test_p9_shear_reference_invariance():
    pitch, L, T = 0.3e-3, 7, 256
    s1 = C / (FS * pitch)
    th = np.arcsin(s1)
    rx = np.array([-th, 0.0, th])
    # grid close to the point so every sample read is far from the record ends
    grid = (12, 10, -0.6e-3, 0.1e-3, 3.5e-3, 0.1e-3)
    w = kksynth.workload_custom("p9", 9, L, pitch, 3, 6.0, T, grid,
                                kksynth.point_phantom([(0.0, 4.0)]))
    ps = schemes.full_product(w.tx_angles, [0, 1, 2], [rx])
    Ba = kk.kk_image(w.rf, w.elem_x, ps, grid, FS, C, rule="advance")
    Br = kk.kk_image(w.rf, w.elem_x, ps, grid, FS, C, rule="retard")
    Bc = kk.kk_image(w.rf, w.elem_x, ps, grid, FS, C, rule="centre")
    assert np.abs(Ba).max() > 0
    assert kk.rel_l2(Br, Ba) <= 1e-10
    assert kk.rel_l2(Bc, Ba) <= 1e-10


# ----------------------------------------------------------------------------
# P10: mirror symmetry (pins the sign conventions of the shear and tau_out)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["vernier", "confocal", "same"])
def test_p10_mirror_symmetry(kind):
    w = kksynth.workload_tiny(seed=31, n_elem=8, n_tx=5, n_samples=96, nx=9, nz=7)
    nx, nz, x0, dx, z0, dz = w.grid
    assert abs(x0 + dx * (nx - 1) / 2) < 1e-15    # symmetric grid
    ps = schemes.scheme(kind, w.tx_angles, 5)
    B = kk.kk_image(w.rf, w.elem_x, ps, w.grid, FS, C)[0]
    Bm = kk.kk_image(w.rf[::-1, ::-1, :].copy(), w.elem_x, ps, w.grid, FS, C)[0]
    assert kk.rel_l2(Bm, B[:, ::-1]) <= 1e-12
    D = kk.das_image(w.rf, w.tx_angles, w.elem_x, w.grid, FS, C)
    Dm = kk.das_image(w.rf[::-1, ::-1, :].copy(), w.tx_angles, w.elem_x, w.grid, FS, C)
    assert kk.rel_l2(Dm, D[:, ::-1]) <= 1e-12


# ----------------------------------------------------------------------------
# P4: point targets focus at their true positions (every scheme and DAS)
# ----------------------------------------------------------------------------
def _peak_offsets(A, grid, points_mm, win=6):
    nx, nz, x0, dx, z0, dz = grid
    out = []
    for (x, z) in points_mm:
        ix = int(round((x * 1e-3 - x0) / dx))
        iz = int(round((z * 1e-3 - z0) / dz))
        lo_x, lo_z = max(ix - win, 0), max(iz - win, 0)
        sub = A[lo_z:iz + win + 1, lo_x:ix + win + 1]
        jz, jx = np.unravel_index(np.argmax(sub), sub.shape)
        out.append((lo_x + jx - ix, lo_z + jz - iz))
    return out


@pytest.mark.parametrize("kind,kw", [("same", {}), ("vernier", {}), ("shifted", {"j": 5}),
                                     ("confocal", {}), ("hybrid", {"js": [0, 2, 5]})])
def test_p4_point_focus_kk(kind, kw):
    w = kksynth.workload_small(speckle=0)
    ps = schemes.scheme(kind, w.tx_angles, 11, **kw)
    B = kk.kk_image(w.rf, w.elem_x, ps, w.grid, FS, C)
    for mode in (["incoherent", "coherent"] if ps.n_groups > 1 else ["coherent"]):
        I = kk.compound(B, mode)
        for off in _peak_offsets(I, w.grid, kksynth.phantom.SMALL_POINTS_MM):
            assert max(abs(off[0]), abs(off[1])) <= 1, (kind, mode, off)


def test_p4_point_focus_das():
    w = kksynth.workload_small(speckle=0)
    D = kk.das_image(w.rf, w.tx_angles, w.elem_x, w.grid, FS, C)
    for off in _peak_offsets(np.abs(D), w.grid, kksynth.phantom.SMALL_POINTS_MM):
        assert max(abs(off[0]), abs(off[1])) <= 1, off


def test_p4_negative_control_planted_shear_sign_defocuses(monkeypatch):
    """Plant a sign mistake in the oracle's shear (a retard instead of an
    advance): P4 must then fail, or it could not see that mistake."""
    w = kksynth.workload_small(speckle=0)
    ps = schemes.scheme("confocal", w.tx_angles, 11)
    good = kk.shear_delays
    monkeypatch.setattr(kk, "shear_delays", lambda *a, **k: -good(*a, **k))
    I = kk.compound(kk.kk_image(w.rf, w.elem_x, ps, w.grid, FS, C), "coherent")
    offs = _peak_offsets(I, w.grid, kksynth.phantom.SMALL_POINTS_MM)
    assert any(max(abs(a), abs(b)) > 1 for a, b in offs)


# ----------------------------------------------------------------------------
# P5: k-space support of the point-spread function, Eq. (kspace): the PSF's
# spectrum sits on k = f (s_i + s_o) / c over the pulse band
# ----------------------------------------------------------------------------
def _kspace_fraction(ps, elem_x, rf, grid, sign=+1.0):
    B = kk.kk_image(rf, elem_x, ps, grid, FS, C)[0]
    nx, nz, x0, dx, z0, dz = grid
    win = np.outer(np.hanning(nz), np.hanning(nx))
    P = np.abs(np.fft.fft2(B * win)) ** 2
    kx = np.fft.fftfreq(nx, dx)
    kz = np.fft.fftfreq(nz, dz)
    mask = np.zeros_like(P, dtype=bool)
    alpha = kksynth.pulse_alpha()
    # pulse amplitude spectrum exp(-pi^2 (f-f0)^2 / alpha) above -40 dB
    half = np.sqrt(np.log(100.0) * alpha) / np.pi
    freqs = np.linspace(kksynth.F0 - half, kksynth.F0 + half, 400)
    th_i, th_o = ps.theta_i(), ps.theta_o()
    for a_i, a_o in zip(th_i, th_o):
        sx = np.sin(a_i) + sign * np.sin(a_o)
        sz = np.cos(a_i) + sign * np.cos(a_o)
        kxs = freqs * sx / C
        kzs = freqs * sz / C
        ix = np.rint(kxs * dx * nx).astype(int) % nx
        iz = np.rint(kzs * dz * nz).astype(int) % nz
        mask[iz, ix] = True
    # dilate by the Hann main lobe (+-2 bins)
    m = mask.copy()
    for sz_ in range(-2, 3):
        for sx_ in range(-2, 3):
            m |= np.roll(np.roll(mask, sz_, axis=0), sx_, axis=1)
    return float(P[m].sum() / P.sum())


def test_p5_kspace_support_of_the_psf():
    lam = C / kksynth.F0
    d = lam / 8
    n = 96
    grid = (n, n, -d * (n - 1) / 2, d, 12e-3 - d * (n - 1) / 2, d)
    w = kksynth.workload_custom("p5", 1, 64, 0.3e-3, 11, 8.0, 512, grid,
                                kksynth.point_phantom([(0.0, 12.0)], amp=1.0))
    for kind, kw in [("vernier", {}), ("shifted", {"j": 5}), ("confocal", {})]:
        ps = schemes.scheme(kind, w.tx_angles, 7, **kw)
        frac = _kspace_fraction(ps, w.elem_x, w.rf, grid)
        assert frac >= 0.99, (kind, frac)
        # the difference-vector reading (s_o - s_i) puts the support elsewhere
        wrong = _kspace_fraction(ps, w.elem_x, w.rf, grid, sign=-1.0)
        assert wrong <= 0.2, (kind, wrong)


# ----------------------------------------------------------------------------
# P7: full-pair KK approximates DAS (Section II-B, after Eq. (KK))
# ----------------------------------------------------------------------------
def test_p7_full_pair_kk_approximates_das():
    lam = C / kksynth.F0
    d = lam / 4
    n = 49                      # odd: the point sits on the centre pixel
    grid = (n, n, -d * (n - 1) / 2, d, 12e-3 - d * (n - 1) / 2, d)
    w = kksynth.workload_custom("p7", 2, 64, 0.3e-3, 11, 8.0, 512, grid,
                                kksynth.point_phantom([(0.0, 12.0)], amp=1.0))
    rx = schemes.even_receive_set(np.deg2rad(35.0), 71)
    ps = schemes.full_product(w.tx_angles, np.arange(11), [rx])
    Bk = np.abs(kk.kk_image(w.rf, w.elem_x, ps, grid, FS, C)[0])
    Bd = np.abs(kk.das_image(w.rf, w.tx_angles, w.elem_x, grid, FS, C))
    assert np.unravel_index(np.argmax(Bk), Bk.shape) == np.unravel_index(np.argmax(Bd), Bd.shape)
    corr = np.corrcoef(Bk.ravel(), Bd.ravel())[0, 1]
    assert corr >= 0.9, corr
