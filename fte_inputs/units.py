"""Unit system of the synthetic inputs: lengths in au, times in s, speeds in au/s,
magnetic field in nT, energies in MeV, momentum in units of m_p c."""
import math

AU_M = 1.495978707e11            # m
C_AU_S = 299792458.0 / AU_M      # speed of light in au/s
MP_C2_MEV = 938.27208816         # proton rest energy, MeV
OMEGA_SUN = 2.67e-6              # synodic rotation rate, 1/s (Sec. 2.3, after Eq. 6)
KMS = 1.0e3 / AU_M               # 1 km/s in au/s


def kinetic_to_p(e_mev):
    """Momentum (m_p c) of a proton of kinetic energy e_mev: p = sqrt(T (T + 2)), T = E/mc^2."""
    t = e_mev / MP_C2_MEV
    return math.sqrt(t * (t + 2.0))
