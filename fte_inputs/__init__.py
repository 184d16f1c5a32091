"""Seeded synthetic inputs for the focused-transport particle pusher.

This package builds the DATA both implementations consume: gridded solar-wind
snapshots (the stand-in for Icarus/EUHFORIA MHD output, Sec. 2.2-2.3), injection
specifications (Sec. 2.3, Eq. 7), transport parameters (Sec. 2.1, Eq. 5) and
observer definitions.  It contains none of the transport method's arithmetic
(no SDE step, no interpolation of the background, no tally): it only evaluates
the synthetic wind models on grid cell centres and takes finite differences of
them, as an MHD code's output post-processor would.
"""
from .units import AU_M, C_AU_S, MP_C2_MEV, OMEGA_SUN, KMS, kinetic_to_p
from .grid import GridSpec, REC, NFIELD, cell_centres
from . import backgrounds, configs

__all__ = [
    "AU_M", "C_AU_S", "MP_C2_MEV", "OMEGA_SUN", "KMS", "kinetic_to_p",
    "GridSpec", "REC", "NFIELD", "cell_centres", "backgrounds", "configs",
]
