"""Units and uniform-electron-gas parameters (oracle; test infrastructure).

Sec. VI.A, Eq. ueg_action: eps_k = hbar^2 k^2 / 2m, V_q = 4 pi e^2 / q^2, density
from r_s.  Reading used throughout: Rydberg units, a0 = 1, hbar^2/2m = 1 (so
m = 1/2) and e^2 = 2, hence eps_k = k^2 - mu and V_q = 8 pi / (q^2 + Lambda)
(Eq. interaction_ct with the screening parameter entering as Lambda = lambda^2).
k_F = (9 pi / 4)^(1/3) / r_s, E_F = k_F^2 = mu_R, T_F = E_F, beta = 1 / T.
"""
import math
from dataclasses import dataclass


@dataclass(frozen=True)
class UEGParams:
    rs: float
    kF: float
    EF: float
    mu: float
    beta: float
    Lambda: float
    kc: float
    kext: float


def ueg_params(rs, T_over_TF, lam_over_kF, kext_over_kF, kc_over_kF=6.0):
    """Physical parameters of one instance from its dimensionless description."""
    kF = (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs
    EF = kF * kF
    beta = 1.0 / (T_over_TF * EF)
    return UEGParams(rs=rs, kF=kF, EF=EF, mu=EF, beta=beta,
                     Lambda=(lam_over_kF * kF) ** 2, kc=kc_over_kF * kF,
                     kext=kext_over_kF * kF)
