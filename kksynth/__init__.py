"""Seeded synthetic inputs for KK / DAS beamforming (input generation only).

This package is shared by the FP64 oracle and the CUDA path.  It builds
phantoms, array geometry, transmit angle sets and RF channel data, and it holds
none of the beamforming method's arithmetic: no far-field decomposition, no
receive-angle schemes, no image formation.  Both sides of every parity test
read the exact bytes produced here.

Workload shapes follow the paper's acquisitions (linear array, plane-wave
transmits evenly spaced over +-theta_max, 5 MHz pulse, ~20 MHz sampling;
Section II-E, Table 1) scaled to the configurations used in the tests and the
benchmark.
"""
from .phantom import (  # noqa: F401
    C_SOUND, FS, F0, BW,
    Phantom, Workload,
    pulse_alpha, pulse_half_window, element_positions, tx_angles_even,
    simulate_rf, add_noise_and_quantise,
    workload_small, workload_large, workload_tiny, workload_custom,
    point_phantom,
    LARGE_WIRES_MM, LARGE_CYSTS_MM,
)
from .images import speckle_images  # noqa: F401
from .volume import (Volume, matrix_elements, tilt_grid, simulate_rf3,  # noqa: F401
                     volume_workload)
