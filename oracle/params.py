"""FP64 reference formulas of the slip boundary scheme (oracle side).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module; only the tests, the smoke check and the CPU-baseline leg of the
benchmark use it.  It shares no code with the CUDA library, which carries its
own host-side precompute.

Every function is the paper's printed closed form written out in plain FP64
(lattice units, delta_x = delta_t = 1, s = sqrt(6/pi)).  Citations name the
paper's section and equation label.
"""
from __future__ import annotations

import math

import numpy as np

S6PI = math.sqrt(6.0 / math.pi)  # sqrt(6/pi), Eq. tKnrela

# D2Q9 lattice, Eq. 3: c_i for i = 0..8 and the weights w_i (Sec. 2).
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6], dtype=np.int64)

# Transformation matrix M of Sec. 2 (Lallemand-Luo ordering
# rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy), as printed.
M = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],
    [-4, -1, -1, -1, -1, 2, 2, 2, 2],
    [4, -2, -2, -2, -2, 1, 1, 1, 1],
    [0, 1, 0, -1, 0, 1, -1, -1, 1],
    [0, -2, 0, 2, 0, 1, -1, -1, 1],
    [0, 0, 1, 0, -1, 1, 1, -1, -1],
    [0, 0, -2, 0, 2, 1, 1, -1, -1],
    [0, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 1, -1, 1, -1],
], dtype=np.float64)


# --------------------------------------------------------------------------
# relaxation times and slip coefficients (Sec. 2, Sec. 4)
# --------------------------------------------------------------------------

def tau_s_from_kn(Kn: float, H: float) -> float:
    """Eq. tKnrela: tau_s = 1/2 + sqrt(6/pi) Kn H / delta_x."""
    return 0.5 + S6PI * Kn * H


def slip_coefficients(sigma: float = 1.0) -> tuple[float, float]:
    """Sec. 4: L1 = (2 - sigma)(1 - 0.1817 sigma)/sigma, L2 = 1/pi + L1^2/2."""
    L1 = (2.0 - sigma) * (1.0 - 0.1817 * sigma) / sigma
    L2 = 1.0 / math.pi + 0.5 * L1 * L1
    return L1, L2


def viscosity(tau_s: float) -> float:
    """Eq. EqViscos with c_s^2 = 1/3, delta_t = 1."""
    return (tau_s - 0.5) / 3.0


# --------------------------------------------------------------------------
# Sec. 3.B: free parameter, combination parameter, uniform tau_q
# --------------------------------------------------------------------------

def l_of_gamma(gamma, tau_s, L1, E):
    """Eq. Eqexlva: l(gamma) that makes tau_q independent of gamma."""
    g = np.asarray(gamma, dtype=np.float64)
    return (S6PI * g * g + g * (2 * tau_s - 1) * (L1 + S6PI)) / (S6PI * (2 * tau_s - 1)) + E


def r_general(l, tau_s, L1):
    """Eq. SliCoeffrtsr: r for any free parameter l."""
    l = np.asarray(l, dtype=np.float64)
    num = S6PI * tau_s * (1 + l)
    return num / (L1 * (2 * tau_s - 1) + num)


def tau_q_general(l, gamma, tau_s, L1, L2):
    """Eq. SliCoeffrtstq: tau_q for any (l, gamma)."""
    l = np.asarray(l, dtype=np.float64)
    g = np.asarray(gamma, dtype=np.float64)
    a = 2 * tau_s - 1
    num = (L1 * a * (2 * tau_s * (6 * g - 1) + 1)
           + S6PI * tau_s * (L2 * math.pi * a * a + 12 * g * g + 2 * a * (6 * g - 6 * l - 1)))
    den = 4 * a * (2 * S6PI * tau_s + L1 * a)
    return num / den


def r_of_gamma(gamma, tau_s, L1, E):
    """Eq. NSliCoertsr: r once l follows Eq. Eqexlva."""
    g = np.asarray(gamma, dtype=np.float64)
    a = 2 * tau_s - 1
    common = S6PI * tau_s * (g * g + g * a + (1 + E) * a)
    return (L1 * tau_s * g * a + common) / (L1 * a * ((2 + g) * tau_s - 1) + common)


def tau_q_uniform(tau_s, L1, L2, E):
    """Eq. NSliCoertstq: the gamma-independent tau_q."""
    a = 2 * tau_s - 1
    num = a * (tau_s * math.sqrt(6 * math.pi) * L2 - L1) - 2 * S6PI * tau_s * (1 + 6 * E)
    den = 8 * S6PI * tau_s + 4 * L1 * a
    return num / den


def E_for_bgk(tau_s, L1, L2):
    """Sec. 3.B, BGK remark: the E for which Eq. NSliCoertstq gives
    tau_q = tau_s (Eq. NSliCoertstq solved for E)."""
    a = 2 * tau_s - 1
    return ((a * (tau_s * math.sqrt(6 * math.pi) * L2 - L1) - 2 * S6PI * tau_s
             - tau_s * (8 * S6PI * tau_s + 4 * L1 * a)) / (12 * S6PI * tau_s))


def E_upper_bound(tau_s, L1, L2):
    """Eq. EqECond: tau_q > 1/2 requires E below this value."""
    return ((math.pi * tau_s * L2 - 3 * math.sqrt(math.pi / 6) * L1) * (2 * tau_s - 1)
            / (12 * tau_s) - 0.5)


def r_halfway(tau_s, L1):
    """Eq. SliCoeffHar (= Eq. SliCoeffrtsrD): halfway DBB / l = 0 scheme."""
    return S6PI * tau_s / (L1 * (2 * tau_s - 1) + S6PI * tau_s)


def tau_q_l0(gamma, tau_s, L1, L2):
    """Eq. SliCoeffrtstqrD: tau_q of the l = 0 scheme at a fixed gamma."""
    g = gamma
    a = 2 * tau_s - 1
    num = (L1 * a * (2 * tau_s * (6 * g - 1) + 1)
           + S6PI * tau_s * (L2 * math.pi * a * a + 12 * g * g + 2 * a * (6 * g - 1)))
    return num / (4 * a * (2 * S6PI * tau_s + L1 * a))


def tau_q_halfway(tau_s, L1, L2):
    """Eq. SliCoeffHata: tau_q of the halfway DBB scheme."""
    a = 2 * tau_s - 1
    num = L1 * a * (4 * tau_s + 1) + S6PI * tau_s * (L2 * math.pi * a * a + 4 * a + 3)
    return num / (4 * a * (2 * S6PI * tau_s + L1 * a))


# --------------------------------------------------------------------------
# Sec. 3.B analysis of the unidirectional channel
# --------------------------------------------------------------------------

def wall_recursion_coefficients(r, l, gamma, tau_s, tau_q):
    """Eq. u1u0Coeff: u_1 = A u_0 + B a dt + C u_w at the wall row."""
    d = (1 + l) * (1 - r) * tau_s + 2 * r * gamma
    A = ((1 + l) * (1 - r) * tau_s + 2 * r * (1 + gamma)) / d
    C = -2 * r / d
    B = (((1 + r + l - l * r) * (1 + 4 * tau_q - 8 * tau_s - 8 * tau_q * tau_s)
          + 12 * r * ((2 * gamma - l) * (2 * tau_s - 1) + (1 - 2 * gamma) * tau_s))
         / (2 * d * (2 * tau_s - 1)))
    return A, B, C


def wall_recursion_coefficients_printed(r, l, gamma, tau_s, tau_q):
    """The wall relation u_1 = A' u_0 + B' a dt + C' u_w of the same channel
    analysis (Sec. 3.B, Eqs. EqMicroBound -> NumerSana) with the Maxwell part
    of Eq. EqNewBDSC evaluated as printed, f_i^eq(rho_f, u_b), instead of at
    the fluid velocity of x_f.

    Route (linear in u and a, Eq. EqAssumpt): only the x-odd combinations
    f_1 - f_3, f_5 - f_6, f_8 - f_7 of a row carry the flow; the difference
    of Eq. EqNewBDSC for i = 5 and i = 6 at the wall row contributes
    (1 - r) u_d / 6 from the Maxwell part, with u_d = u_0 in the reading
    under which Eq. u1u0Coeff holds and u_d = u_w as printed.  Eliminating the
    shear moments of rows 0 and 1 gives Eq. u1u0Coeff for u_d = u_0 and, for
    u_d = u_w, the same B with
        A' = A + (1 + l)(1 - r) / d,   C' = 1 - A',
        d  = (1 + l)(1 - r) tau_s + 2 r gamma.
    A' + C' = 1: a uniform flow at the wall speed is steady."""
    A, B, _ = wall_recursion_coefficients(r, l, gamma, tau_s, tau_q)
    d = (1 + l) * (1 - r) * tau_s + 2 * r * gamma
    Ap = A + (1 + l) * (1 - r) / d
    return Ap, B, 1 - Ap


def slip_velocity_numeric(r, l, gamma, tau_s, tau_q, H):
    """Eq. EqMiSlip: U_s = u_s / u_c of the scheme for any parameters
    (delta_x = 1, channel width H)."""
    D = (12 * gamma ** 2 + 12 * gamma * (tau_s - 1)
         + (2 * tau_s - 1) * (4 * l * tau_q - 1 - 4 * tau_q)
         - l * (11 * (2 * tau_s - 1) + 12 * gamma * tau_s))
    return (2 * (1 + l) * (1 - r) / r * tau_s / H
            - ((1 + l) * (1 + 4 * tau_q - 2 * tau_s + 12 * gamma * tau_s - 8 * tau_s * tau_q)
               + r * D) / (3 * r) / H ** 2)


def slip_velocity_kn(r, l, gamma, tau_s, tau_q, Kn):
    """Eq. NumeriSlip: the same slip velocity written with Kn."""
    a = 2 * tau_s - 1
    K = (a * (1 + r + l + 11 * l * r) + 12 * gamma * (r + tau_s * (l * r - l - r - 1))
         - 12 * r * gamma ** 2 - 4 * tau_q * a * (l * r - l - r - 1))
    return (4 * (1 - r) * (1 + l) * tau_s / (r * a) * S6PI * Kn
            + 8 / math.pi * K / (r * a * a) * Kn * Kn)


def slip_velocity_physical(L1, L2, Kn):
    """Eq. PhyscPoiSlip: U_s = 4 L1 Kn + 8 L2 Kn^2."""
    return 4 * L1 * Kn + 8 * L2 * Kn * Kn


def poiseuille_profile(y, H, u_c, U_s, u_w=0.0):
    """Eq. OrSnumve / numvelo: u = 4 u_c y/H (1 - y/H) + u_w + u_s."""
    y = np.asarray(y, dtype=np.float64)
    return 4 * u_c * y / H * (1 - y / H) + u_w + U_s * u_c


def couette_profile(r, R1, R2, omega1, omega2, lam, sigma1=1.0, sigma2=1.0):
    """Eq. EqAnaMicro with Eq. EqAnaPraMicro: u_theta(r) between rotating
    cylinders with first-order Maxwell slip."""
    r = np.asarray(r, dtype=np.float64)
    Mc = (1 - (2 - sigma2) / sigma2 * 2 * lam / R2) / R2 ** 2
    Nc = (1 + (2 - sigma1) / sigma1 * 2 * lam / R1) / R1 ** 2
    return (Mc * omega1 - Nc * omega2) / (Mc - Nc) * r + (omega1 - omega2) / (Nc - Mc) / r


# --------------------------------------------------------------------------
# per-case parameter set and per-link (r, l, gamma)
# --------------------------------------------------------------------------

class Parameters:
    """All FP64 parameters of one case.

    E policy (the paper gives E = -0.65 and -0.68 and the bound of
    Eq. EqECond but no rule): E = min(-0.65, E_max - 0.1).  The clamp of
    Sec. 3.B: l := 0 where Eq. Eqexlva gives l < -0.4, and r then follows
    Eq. SliCoeffrtsr with the l actually used (identical to Eq. NSliCoertsr
    where no clamp applies).

    `bgk=True` takes the BGK reading of Sec. 3.B: every relaxation time
    equals tau_s and E solves Eq. NSliCoertstq for tau_q = tau_s.

    `l_mode` selects the free parameter: "paper" (Eq. Eqexlva), "zero",
    "gamma", "2gamma", "gamma2", "gamma2+gamma" (the alternatives of
    Sec. 4) or a float (a fixed l).  `r_fixed` and `tau_q_fixed` replace the
    tuned values (used for the untuned sweeps of Sec. 4.A.1).
    """

    def __init__(self, Kn, H, sigma=1.0, L1=None, L2=None, E=None, l_clamp=-0.4,
                 tau_rho=1.0, tau_j=1.0, tau_e=1.1, tau_eps=1.2, l_mode="paper",
                 r_fixed=None, tau_q_fixed=None, tau_s=None, bgk=False):
        self.Kn = float(Kn)
        self.H = float(H)
        self.tau_s = tau_s_from_kn(Kn, H) if tau_s is None else float(tau_s)
        dL1, dL2 = slip_coefficients(sigma)
        self.L1 = dL1 if L1 is None else float(L1)
        self.L2 = dL2 if L2 is None else float(L2)
        self.E_max = E_upper_bound(self.tau_s, self.L1, self.L2)
        self.E = min(-0.65, self.E_max - 0.1) if E is None else float(E)
        if bgk:
            # BGK (Sec. 3.B): one relaxation time tau_s for every moment and
            # the E that makes the uniform tau_q equal to it
            self.E = E_for_bgk(self.tau_s, self.L1, self.L2)
            tau_rho = tau_j = tau_e = tau_eps = self.tau_s
        self.l_clamp = l_clamp
        self.l_mode = l_mode
        self.r_fixed = r_fixed
        if tau_q_fixed is not None:
            self.tau_q = float(tau_q_fixed)
        else:
            self.tau_q = tau_q_uniform(self.tau_s, self.L1, self.L2, self.E)
        self.tau_rho, self.tau_j, self.tau_e, self.tau_eps = tau_rho, tau_j, tau_e, tau_eps

    def relaxation_times(self) -> np.ndarray:
        """Diagonal of S^-1 in the moment order of M (Sec. 2)."""
        return np.array([self.tau_rho, self.tau_e, self.tau_eps, self.tau_j, self.tau_q,
                         self.tau_j, self.tau_q, self.tau_s, self.tau_s])

    def relaxation_times_d3q19(self) -> np.ndarray:
        """Relaxation times of the 19 D3Q19 moments in the order of the 3-D
        oracle's basis (rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx,
        3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z).  The paper
        fixes only tau_s (stress) and tau_q (energy flux) through its
        two-dimensional analysis.  Carried out for D3Q19 (flow u_x(z) between
        walls normal to z), that analysis reaches the same wall relation
        Eq. u1u0Coeff exactly when the third-order moments m relax with
        tau_q, so m takes tau_q; the fourth-order pi take tau_eps."""
        return np.array([self.tau_rho, self.tau_e, self.tau_eps, self.tau_j, self.tau_q,
                         self.tau_j, self.tau_q, self.tau_j, self.tau_q, self.tau_s, self.tau_eps,
                         self.tau_s, self.tau_eps, self.tau_s, self.tau_s, self.tau_s, self.tau_q,
                         self.tau_q, self.tau_q])

    def link_l(self, gamma) -> np.ndarray:
        g = np.asarray(gamma, dtype=np.float64)
        m = self.l_mode
        if m == "paper":
            l = l_of_gamma(g, self.tau_s, self.L1, self.E)
            return np.where(l < self.l_clamp, 0.0, l)
        if m == "zero":
            return np.zeros_like(g)
        if m == "gamma":
            return g.copy()
        if m == "2gamma":
            return 2 * g
        if m == "gamma2":
            return g * g
        if m == "gamma2+gamma":
            return g * g + g
        return np.full_like(g, float(m))

    def link_r(self, l) -> np.ndarray:
        l = np.asarray(l, dtype=np.float64)
        if self.r_fixed is not None:
            return np.full_like(l, float(self.r_fixed))
        return r_general(l, self.tau_s, self.L1)

    def per_link(self, gamma):
        """(r, l) per link for distance ratios `gamma`."""
        l = self.link_l(gamma)
        return self.link_r(l), l
