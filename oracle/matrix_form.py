"""Single-node PRC-LBM collision in matrix form (oracle-B), numpy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

This is a second, independent statement of the collision, written from the
main text of arXiv:2208.03562 rather than from Appendix A:

* moment bases: Q (Eq. Q-momentbasis) built from the rectangular velocities of
  Eq. 3, P (Eq. P-momentbasis) from the square ones, S (Eq. S-matrix), and the
  combination matrix B of Eq. TandQrelation (T = B Q, with T from Eqs. 7-8);
* the frame-shift matrix F(u) exactly as printed in Eq. Fmatrix, which acts on
  moments in the combined (k2s, k2d) basis of T, with F^-1 = F(-u) (Sec. 4.2);
* equilibria Eq. 12/14 in the combined basis, extended by the corrections of
  Eqs. 30-31 with the coefficients of Eqs. 38-40 and the prefactors of
  Eq. prefactors (numbered 3, 4, 5 as in Sec. 3);
* strain rates from Eqs. 43, 45, 46 and 48;
* sources Eq. 13-central; relaxation matrix Eq. 11 (zero rates for the
  conserved moments).

The post-collision populations are then

    f~ = P^-1 S^-1 B^-1 F(-u) [ n^c + Lambda (n^c,eq - n^c) + (I - Lambda/2) Psi^c ]

with n^c = F(u) B S P f, which is Eq. 10-equivalent-centralmoment written with
the combined-basis F.  Typos read as in the oracle's header (A6: lambda_4x and
lambda_5x for the repeated symbols of Eq. 31).
"""
import numpy as np

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
EYB = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)
CS_STAR2 = 1.0 / 3.0  # Eq. 1


def monomial_basis(ex: np.ndarray, ey: np.ndarray) -> np.ndarray:
    """Rows |1>, |ex>, |ey>, |ex^2>, |ey^2>, |ex ey>, |ex^2 ey>, |ex ey^2>,
    |ex^2 ey^2> (the bare basis of Eq. Q-momentbasis / Eq. P-momentbasis)."""
    return np.array([
        np.ones(9), ex, ey, ex ** 2, ey ** 2, ex * ey, ex ** 2 * ey, ex * ey ** 2, ex ** 2 * ey ** 2,
    ])


def T_basis(ex: np.ndarray, ey: np.ndarray) -> np.ndarray:
    """Eqs. 7-8: the combined non-orthogonal basis T."""
    return np.array([
        np.ones(9), ex, ey, ex ** 2 + ey ** 2, ex ** 2 - ey ** 2, ex * ey, ex ** 2 * ey, ex * ey ** 2,
        ex ** 2 * ey ** 2,
    ])


def P_matrix() -> np.ndarray:
    return monomial_basis(EX, EYB)


def Q_matrix(r: float) -> np.ndarray:
    return monomial_basis(EX, r * EYB)


def S_matrix(r: float) -> np.ndarray:
    return np.diag([1, 1, r, 1, r ** 2, r, r, r ** 2, r ** 2]).astype(np.float64)


def B_matrix() -> np.ndarray:
    B = np.eye(9)
    B[3, 3], B[3, 4] = 1.0, 1.0
    B[4, 3], B[4, 4] = 1.0, -1.0
    return B


def F_matrix(ux: float, uy: float) -> np.ndarray:
    """Eq. Fmatrix, row by row, combined-basis ordering
    (k00, k10, k01, k2s, k2d, k11, k21, k12, k22)."""
    return np.array([
        [1, 0, 0, 0, 0, 0, 0, 0, 0],
        [-ux, 1, 0, 0, 0, 0, 0, 0, 0],
        [-uy, 0, 1, 0, 0, 0, 0, 0, 0],
        [ux ** 2 + uy ** 2, -2 * ux, -2 * uy, 1, 0, 0, 0, 0, 0],
        [ux ** 2 - uy ** 2, -2 * ux, 2 * uy, 0, 1, 0, 0, 0, 0],
        [ux * uy, -uy, -ux, 0, 0, 1, 0, 0, 0],
        [-ux ** 2 * uy, 2 * ux * uy, ux ** 2, -0.5 * uy, -0.5 * uy, -2 * ux, 1, 0, 0],
        [-ux * uy ** 2, uy ** 2, 2 * ux * uy, -0.5 * ux, 0.5 * ux, -2 * uy, 0, 1, 0],
        [ux ** 2 * uy ** 2, -2 * ux * uy ** 2, -2 * ux ** 2 * uy, 0.5 * (ux ** 2 + uy ** 2),
         0.5 * (uy ** 2 - ux ** 2), 4 * ux * uy, -2 * uy, -2 * ux, 1],
    ], dtype=np.float64)


def omega_nu_of(nu: float, gamma: float, r: float) -> float:
    """Eq. transport-coefficients solved for the shear rate."""
    q = min(1.0, r)
    return 1.0 / (nu / (gamma * q * q * CS_STAR2) + 0.5)


def equilibrium_populations(r, gamma, rho, ux, uy):
    """f^eq = Q^-1 m^eq with m^eq from Eq. 12 (bare ordering)."""
    q = min(1.0, r)
    c2 = q * q * CS_STAR2
    g = gamma
    meq = np.array([
        rho, rho * ux, rho * uy,
        c2 * rho + rho * ux ** 2 / g, c2 * rho + rho * uy ** 2 / g, rho * ux * uy / g,
        rho * (c2 + ux ** 2 / g ** 2) * uy, rho * (c2 + uy ** 2 / g ** 2) * ux,
        rho * c2 ** 2 + rho * c2 * (ux ** 2 + uy ** 2) + rho * ux ** 2 * uy ** 2,
    ])
    return np.linalg.solve(Q_matrix(r), meq)


def collide(f, r, gamma, omega_nu, dxrho=0.0, dyrho=0.0, fx=0.0, fy=0.0,
            omega_3=1.0, omega_6=1.0, omega_7=1.0, omega_8=1.0, corrections=True):
    """Post-collision populations of one node (matrix form). Returns (f~, diag)
    with diag = (rho, u_x, u_y, d_x u_x, d_y u_y)."""
    f = np.asarray(f, dtype=np.float64)
    q = min(1.0, r)
    c2 = q * q * CS_STAR2  # q^2 c_s*^2
    g = gamma
    w3, w4, w5 = omega_3, omega_nu, omega_nu
    P, S, B = P_matrix(), S_matrix(r), B_matrix()

    n = B @ S @ P @ f  # combined raw moments, n = T f
    rho = n[0]
    ux = (n[1] + fx / (2 * g)) / rho
    uy = (n[2] + fy / (2 * g)) / rho
    nc = F_matrix(ux, uy) @ n

    # Eq. prefactors
    M3 = rho * ((4 / g ** 2 - 1 / g) * ux ** 2 + (1 / g ** 2 - 1 / g) * uy ** 2)
    N3 = rho * ((4 / g ** 2 - 1 / g) * uy ** 2 + (1 / g ** 2 - 1 / g) * ux ** 2)
    M4 = rho * ((4 / g ** 2 - 1 / g) * ux ** 2 - (1 / g ** 2 - 1 / g) * uy ** 2)
    N4 = rho * (-(4 / g ** 2 - 1 / g) * uy ** 2 + (1 / g ** 2 - 1 / g) * ux ** 2)

    corr = np.zeros(9)
    dxux = dyuy = 0.0
    if corrections:
        # Eq. 43
        A = 0.5 * ((2 / g + 1) * c2 - 1) * ux
        Bc = 0.5 * ((2 / g + 1) * c2 - r ** 2) * uy
        e3 = -A * dxrho - Bc * dyrho
        e4 = -A * dxrho + Bc * dyrho
        # Eq. 45
        R3 = nc[3] - 2 * c2 * rho - (1 / g - 1) * (ux ** 2 + uy ** 2) * rho + e3
        R4 = nc[4] - (1 / g - 1) * (ux ** 2 - uy ** 2) * rho + e4
        # Eq. 46
        C3x = -2 * c2 / w3 * rho + M3 / 2 + 0.5 * (3 * c2 - 1) * rho
        C3y = -2 * c2 / w3 * rho + N3 / 2 + 0.5 * (3 * c2 - r ** 2) * rho
        C4x = -2 * c2 / w4 * rho + M4 / 2 + 0.5 * (3 * c2 - 1) * rho
        C4y = 2 * c2 / w4 * rho + N4 / 2 - 0.5 * (3 * c2 - r ** 2) * rho
        # Eq. 47-48: solve the 2x2 system
        dxux, dyuy = np.linalg.solve(np.array([[C3x, C3y], [C4x, C4y]]), np.array([R3, R4]))
        # Eqs. 38-40
        t3, t4, t5 = 1 / w3 - 0.5, 1 / w4 - 0.5, 1 / w5 - 0.5
        th3x = -(M3 + (3 * c2 - 1) * rho) * t3
        th3y = -(N3 + (3 * c2 - r ** 2) * rho) * t3
        la3x = -((2 / g + 1) * c2 - 1) * t3 * ux
        la3y = -((2 / g + 1) * c2 - r ** 2) * t3 * uy
        th4x = -(M4 + (3 * c2 - 1) * rho) * t4
        th4y = +(N4 - (3 * c2 - r ** 2) * rho) * t4
        la4x = -((2 / g + 1) * c2 - 1) * t4 * ux
        la4y = +((2 / g + 1) * c2 - r ** 2) * t4 * uy
        th5x = -(1 / g ** 2 - 1 / g) * t5 * rho * ux * uy
        th5y = -(1 / g ** 2 - 1 / g) * t5 * rho * ux * uy
        la5x = -(1 / g - 1) * t5 * c2 * uy
        la5y = -(1 / g - 1) * t5 * c2 * ux
        # Eq. 31
        corr[3] = th3x * dxux + th3y * dyuy + la3x * dxrho + la3y * dyrho
        corr[4] = th4x * dxux - th4y * dyuy + la4x * dxrho + la4y * dyrho
        corr[5] = th5x * dxux + th5y * dyuy + la5x * dxrho + la5y * dyrho

    # Eq. 14 in the combined basis, plus Eq. 30 (dt = 1)
    a = 1 / g ** 2 - 3 / g + 2
    nceq = np.array([
        rho, 0.0, 0.0,
        2 * c2 * rho + (1 / g - 1) * rho * (ux ** 2 + uy ** 2),
        (1 / g - 1) * rho * (ux ** 2 - uy ** 2),
        (1 / g - 1) * rho * ux * uy,
        a * rho * ux ** 2 * uy, a * rho * ux * uy ** 2, c2 ** 2 * rho,
    ]) + corr

    # Eq. 13-central in the combined basis
    h = 1 / g ** 2 - 1 / g
    s20, s02 = h * 2 * fx * ux, h * 2 * fy * uy
    psi = np.array([0.0, fx / g, fy / g, s20 + s02, s20 - s02, h * (fx * uy + fy * ux), 0.0, 0.0, 0.0])

    Lam = np.diag([0.0, 0.0, 0.0, w3, w4, w5, omega_6, omega_7, omega_8])
    nct = nc + Lam @ (nceq - nc) + (np.eye(9) - Lam / 2) @ psi
    ft = np.linalg.inv(P) @ np.linalg.inv(S) @ np.linalg.inv(B) @ F_matrix(-ux, -uy) @ nct
    return ft, np.array([rho, ux, uy, dxux, dyuy])


def collide_raw(f, r, gamma, omega_nu, dxrho=0.0, dyrho=0.0, fx=0.0, fy=0.0,
                omega_3=1.0, omega_6=1.0, omega_7=1.0, omega_8=1.0, corrections=True):
    """PRNR-LBM collision of one node, as the matrix product of
    Eq. 10-equivalent:

        f~ = P^-1 S^-1 [ m + B^-1 Lambda (B m^eq - B m) + B^-1 (I - Lambda/2) B Phi ]

    with m = S P f, the raw equilibria of Eq. 12 (second order extended by the
    corrections of Eqs. 30-31 with the coefficients of Eqs. 38-40), the raw
    sources of Eq. 13 and Lambda of Eq. 11. The strain rates of the corrections
    come from Eq. 45, as in the central scheme. Returns (f~, diag)."""
    f = np.asarray(f, dtype=np.float64)
    q = min(1.0, r)
    c2 = q * q * CS_STAR2
    g = gamma
    P, S, B = P_matrix(), S_matrix(r), B_matrix()
    m = S @ P @ f
    n = B @ m
    rho = n[0]
    ux = (n[1] + fx / (2 * g)) / rho
    uy = (n[2] + fy / (2 * g)) / rho
    # the correction terms (second order only) are the central scheme's: the
    # difference of the two equilibria in the combined basis at order two
    _, diag = collide(f, r, gamma, omega_nu, dxrho, dyrho, fx, fy, omega_3, omega_6, omega_7, omega_8,
                      corrections)
    corr = _corrections(rho, ux, uy, diag[3], diag[4], dxrho, dyrho, r, g, c2, omega_3, omega_nu) \
        if corrections else np.zeros(9)
    meq = np.array([
        rho, rho * ux, rho * uy,
        2 * c2 * rho + rho * (ux ** 2 + uy ** 2) / g,
        rho * (ux ** 2 - uy ** 2) / g,
        rho * ux * uy / g,
        rho * (c2 + ux ** 2 / g ** 2) * uy,
        rho * (c2 + uy ** 2 / g ** 2) * ux,
        rho * c2 ** 2 + rho * c2 * (ux ** 2 + uy ** 2) + rho * ux ** 2 * uy ** 2,
    ]) + corr
    s20, s02 = 2 * fx * ux / g ** 2, 2 * fy * uy / g ** 2
    phi = np.array([0.0, fx / g, fy / g, s20 + s02, s20 - s02, (fx * uy + fy * ux) / g ** 2, 0.0, 0.0, 0.0])
    Lam = np.diag([0.0, 0.0, 0.0, omega_3, omega_nu, omega_nu, omega_6, omega_7, omega_8])
    Bi = np.linalg.inv(B)
    mt = m + Bi @ Lam @ (meq - n) + Bi @ (np.eye(9) - Lam / 2) @ phi
    ft = np.linalg.inv(P) @ np.linalg.inv(S) @ mt
    return ft, diag


def _corrections(rho, ux, uy, dxux, dyuy, dxrho, dyrho, r, g, c2, w3, w4):
    """Eq. 31 with the coefficients of Eqs. 38-40 (combined basis, second order)."""
    w5 = w4
    M3 = rho * ((4 / g ** 2 - 1 / g) * ux ** 2 + (1 / g ** 2 - 1 / g) * uy ** 2)
    N3 = rho * ((4 / g ** 2 - 1 / g) * uy ** 2 + (1 / g ** 2 - 1 / g) * ux ** 2)
    M4 = rho * ((4 / g ** 2 - 1 / g) * ux ** 2 - (1 / g ** 2 - 1 / g) * uy ** 2)
    N4 = rho * (-(4 / g ** 2 - 1 / g) * uy ** 2 + (1 / g ** 2 - 1 / g) * ux ** 2)
    t3, t4, t5 = 1 / w3 - 0.5, 1 / w4 - 0.5, 1 / w5 - 0.5
    th3x = -(M3 + (3 * c2 - 1) * rho) * t3
    th3y = -(N3 + (3 * c2 - r ** 2) * rho) * t3
    la3x = -((2 / g + 1) * c2 - 1) * t3 * ux
    la3y = -((2 / g + 1) * c2 - r ** 2) * t3 * uy
    th4x = -(M4 + (3 * c2 - 1) * rho) * t4
    th4y = +(N4 - (3 * c2 - r ** 2) * rho) * t4
    la4x = -((2 / g + 1) * c2 - 1) * t4 * ux
    la4y = +((2 / g + 1) * c2 - r ** 2) * t4 * uy
    th5x = -(1 / g ** 2 - 1 / g) * t5 * rho * ux * uy
    th5y = -(1 / g ** 2 - 1 / g) * t5 * rho * ux * uy
    la5x = -(1 / g - 1) * t5 * c2 * uy
    la5y = -(1 / g - 1) * t5 * c2 * ux
    corr = np.zeros(9)
    corr[3] = th3x * dxux + th3y * dyuy + la3x * dxrho + la3y * dyrho
    corr[4] = th4x * dxux - th4y * dyuy + la4x * dxrho + la4y * dyrho
    corr[5] = th5x * dxux + th5y * dyuy + la5x * dxrho + la5y * dyrho
    return corr
