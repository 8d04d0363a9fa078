"""Physical constants and unit conversions of the oracle (CODATA 2018).

Working units: Angstrom, amu, eV, K, ps.  Force constants in eV/A^n, masses
in amu, so an eigenvalue of the dynamical matrix is in eV/(A^2 amu); EV_A2_AMU
converts it to ps^-2 (angular frequency squared).
"""

import math

EV_J = 1.602176634e-19          # J per eV
AMU_KG = 1.66053906660e-27      # kg per amu
ANG_M = 1e-10                   # m per Angstrom
HBAR_JS = 1.054571817e-34       # J s
KB_JK = 1.380649e-23            # J / K

#: 1 eV/(A^2 amu) expressed in ps^-2
EV_A2_AMU = EV_J / (ANG_M ** 2 * AMU_KG) * 1e-24
#: hbar in eV ps
HBAR_EVPS = HBAR_JS / EV_J * 1e12
#: k_B in eV / K
KB_EVK = KB_JK / EV_J

TWO_PI = 2.0 * math.pi
