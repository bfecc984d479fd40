"""Receive-angle schemes and (transmit, receive) pair sets -- oracle side.

TEST INFRASTRUCTURE (see ``oracle/__init__``).  Written from Section II-C and
II-D of the paper; angles are in radians, FP64.

Receive index convention.  The paper writes o = -floor(M/2) .. floor(M/2),
which has M members only for odd M (every M the paper uses is odd).  For even M
this oracle takes o in {-(M-1)/2, ..., (M-1)/2} in unit steps (half-integers),
identical to the paper for odd M; in Eq. (confocal) the shift term then uses
floor(|o|).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def receive_offsets(M: int) -> np.ndarray:
    """o = -(M-1)/2 .. (M-1)/2 in unit steps (Section II-C, after Fig. 2)."""
    if M < 1:
        raise ValueError("M must be >= 1")
    return np.arange(M, dtype=np.float64) - (M - 1) / 2.0


def transmit_spacing(tx_angles) -> float:
    """delta theta_i = 2 theta_max / (N - 1) for evenly spaced transmits (Section II-B)."""
    tx = np.asarray(tx_angles, dtype=np.float64)
    if tx.shape[0] < 2:
        raise ValueError("need at least two transmit angles")
    return float((tx.max() - tx.min()) / (tx.shape[0] - 1))


def rx_same(tx_angles) -> np.ndarray:
    """Receive angles equal to the transmit angles -- the redundant scheme the
    paper calls not optimal (Section II-C, first paragraph)."""
    return np.array(tx_angles, dtype=np.float64)


def rx_shifted(dtheta_i: float, M: int, j: float) -> np.ndarray:
    """Eq. (uniform): theta_o = sgn(o) dtheta_i (2|o|/M + j).  j = 0 is the
    vernier sequence theta_o = 2 o dtheta_i / M of Section II-C."""
    o = receive_offsets(M)
    return np.sign(o) * dtheta_i * (2.0 * np.abs(o) / M + j)


def rx_vernier(dtheta_i: float, M: int) -> np.ndarray:
    """theta_o = 2 o dtheta_i / M (Section II-C): Eq. (uniform) with j = 0."""
    return rx_shifted(dtheta_i, M, 0.0)


def rx_confocal(dtheta_i: float, M: int, N: int) -> np.ndarray:
    """Eq. (confocal): theta_o = sgn(o) dtheta_i (2|o|/M + mod(|o|, floor(N/2)))."""
    half = N // 2
    if half < 1:
        raise ValueError("confocal scheme needs floor(N/2) >= 1")
    o = receive_offsets(M)
    shift = np.mod(np.floor(np.abs(o)), half)
    return np.sign(o) * dtheta_i * (2.0 * np.abs(o) / M + shift)


def strided_subset(n_acquired: int, a: int) -> np.ndarray:
    """Indices of an a-angle transmit subset with a uniform even stride s,
    symmetric about the centre of the acquired set: s is the largest even
    stride with (a-1) s <= n_acquired - 1."""
    if a < 1 or a > n_acquired:
        raise ValueError("bad subset size")
    if a == 1:
        return np.array([(n_acquired - 1) // 2])
    s = (n_acquired - 1) // (a - 1)
    if s % 2:
        s -= 1
    s = max(s, 1)
    start = ((n_acquired - 1) - (a - 1) * s) // 2
    return start + s * np.arange(a)


@dataclasses.dataclass
class PairSet:
    """A KK pair set: P pairs (transmit index, receive index) in J groups.

    ``tx_index`` indexes the acquired transmit angles (rows of the RF data),
    ``rx_angles`` holds every receive angle, ``rx_index`` indexes it.
    """
    tx_angles: np.ndarray     # [N] acquired transmit angles
    rx_angles: np.ndarray     # [M_total]
    tx_index: np.ndarray      # [P] int
    rx_index: np.ndarray      # [P] int
    group: np.ndarray         # [P] int in [0, J)
    n_groups: int
    name: str = ""

    @property
    def n_pairs(self) -> int:
        return int(self.tx_index.shape[0])

    def theta_i(self) -> np.ndarray:
        return self.tx_angles[self.tx_index]

    def theta_o(self) -> np.ndarray:
        return self.rx_angles[self.rx_index]

    def compression_factor(self, n_elem: int) -> float:
        """L / (J M) (Section II-B and after Eq. (incoherent)); M is the number
        of receive angles per group."""
        m_per_group = self.rx_angles.shape[0] / self.n_groups
        return n_elem / (self.n_groups * m_per_group)


def full_product(tx_angles, tx_subset, rx_groups, name="") -> PairSet:
    """Every selected transmit paired with every receive angle of each group
    (one group per entry of ``rx_groups``)."""
    tx_angles = np.asarray(tx_angles, dtype=np.float64)
    tx_subset = np.asarray(tx_subset, dtype=np.int64)
    rx_all, ti, ri, gi = [], [], [], []
    base = 0
    for g, rx in enumerate(rx_groups):
        rx = np.asarray(rx, dtype=np.float64)
        for i in tx_subset:
            for o in range(rx.shape[0]):
                ti.append(int(i))
                ri.append(base + o)
                gi.append(g)
        rx_all.append(rx)
        base += rx.shape[0]
    return PairSet(tx_angles, np.concatenate(rx_all), np.array(ti, dtype=np.int64),
                   np.array(ri, dtype=np.int64), np.array(gi, dtype=np.int64),
                   len(rx_groups), name)


def scheme(kind: str, tx_angles, M: int, j: float = 0, tx_subset=None, js=None) -> PairSet:
    """Pair set for one of the paper's schemes over the transmit subset.

    kind: 'same' | 'vernier' | 'shifted' | 'confocal' | 'hybrid' (groups over
    ``js`` with Eq. (uniform), compounded by Eqs. (coherent)/(incoherent)).
    dtheta_i is the spacing of the transmit subset actually used.
    """
    tx_angles = np.asarray(tx_angles, dtype=np.float64)
    if tx_subset is None:
        tx_subset = np.arange(tx_angles.shape[0])
    tx_subset = np.asarray(tx_subset)
    sub = tx_angles[tx_subset]
    n = sub.shape[0]
    if kind == "same":
        return full_product(tx_angles, tx_subset, [rx_same(sub)], "same")
    dth = transmit_spacing(sub)
    if kind == "vernier":
        return full_product(tx_angles, tx_subset, [rx_vernier(dth, M)], f"vernier{n}x{M}")
    if kind == "shifted":
        return full_product(tx_angles, tx_subset, [rx_shifted(dth, M, j)], f"shifted{n}x{M}j{j}")
    if kind == "confocal":
        return full_product(tx_angles, tx_subset, [rx_confocal(dth, M, n)], f"confocal{n}x{M}")
    if kind == "hybrid":
        js = list(js) if js is not None else [0, n // 4, n // 2]
        return full_product(tx_angles, tx_subset, [rx_shifted(dth, M, jj) for jj in js],
                            f"hybrid{n}x{M}j{'-'.join(str(x) for x in js)}")
    raise ValueError(f"unknown scheme {kind}")


def even_receive_set(theta_max: float, M: int) -> np.ndarray:
    """M receive angles evenly spaced over +-theta_max, endpoints included
    (a full N x M acquisition-like pair set)."""
    if M == 1:
        return np.zeros(1)
    return np.linspace(-theta_max, theta_max, M)


def paraxial_differences(ps: PairSet) -> np.ndarray:
    """Delta theta = theta_o - theta_i for every pair (proportional to k_x in
    the paraxial limit, Section II-C, Fig. 2b)."""
    return ps.theta_o() - ps.theta_i()
