"""Pure-Python brute force of the whole KK / DAS chain for tiny inputs.

Explicit loops, a direct O(T^2) DFT with ``cmath``, no numpy arithmetic.  Used
to catch vectorisation mistakes (transposed operands, wrong axes, wrong
broadcasting) in the numpy/C oracle; it restates the same definitions, so the
oracle's physics is pinned by the other tests, not by this one.
"""
import cmath
import math


def dft_analytic(x):
    """Direct DFT, Hilbert weights, direct inverse of the half spectrum."""
    T = len(x)
    F = T // 2
    X = []
    for k in range(F):
        acc = 0j
        for t in range(T):
            acc += x[t] * cmath.exp(-2j * math.pi * k * t / T)
        X.append(acc * (1.0 if k == 0 else 2.0))
    return X


def idft_half(Y, T):
    out = []
    for t in range(T):
        acc = 0j
        for k in range(len(Y)):
            acc += Y[k] * cmath.exp(2j * math.pi * k * t / T)
        out.append(acc / T)
    return out


def xref(elem_x, th):
    if th > 0:
        return max(elem_x)
    if th < 0:
        return min(elem_x)
    return 0.0


def lerp(y, s):
    T = len(y)
    k = math.floor(s)
    if k < 0 or k + 1 > T - 1:
        return 0j
    f = s - k
    return (1 - f) * y[k] + f * y[k + 1]


def kk_chain(rf, elem_x, tx_angles, pairs, groups, J, pix, fs, c):
    """rf: nested lists [N][L][T]; pairs: list of (i, theta_o); pix: list of (x, z)."""
    T = len(rf[0][0])
    L = len(elem_x)
    spectra = {}
    ys = []
    for (i, th) in pairs:
        if i not in spectra:
            spectra[i] = [dft_analytic(rf[i][l]) for l in range(L)]
        Xi = spectra[i]
        xr = xref(elem_x, th)
        Y = []
        for k in range(T // 2):
            acc = 0j
            for l in range(L):
                d = (xr - elem_x[l]) * math.sin(th) / c
                acc += Xi[l][k] * cmath.exp(2j * math.pi * k * fs * d / T)
            Y.append(acc)
        ys.append(idft_half(Y, T))
    out = [[0j for _ in pix] for _ in range(J)]
    for q, (x, z) in enumerate(pix):
        for p, (i, th) in enumerate(pairs):
            ti = tx_angles[i]
            tau = (x * math.sin(ti) + z * math.cos(ti)) / c
            tau += ((x - xref(elem_x, th)) * math.sin(th) + z * math.cos(th)) / c
            out[groups[p]][q] += lerp(ys[p], fs * tau)
    return out


def das_chain(rf, elem_x, tx_angles, pix, fs, c):
    T = len(rf[0][0])
    N, L = len(rf), len(elem_x)
    y = [[idft_half(dft_analytic(rf[i][l]), T) for l in range(L)] for i in range(N)]
    out = []
    for (x, z) in pix:
        acc = 0j
        for i in range(N):
            ti = tx_angles[i]
            for l in range(L):
                tau = (x * math.sin(ti) + z * math.cos(ti)) / c
                tau += math.sqrt((x - elem_x[l]) ** 2 + z * z) / c
                acc += lerp(y[i][l], fs * tau)
        out.append(acc)
    return out
