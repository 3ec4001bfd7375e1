"""Closed-form steady solutions used to pin the oracle (test infrastructure only).

Every formula here is derived from the governing equation the paper's LBM
recovers (Eq. 7 with the momentum, convection-diffusion and induction
equations of Sec. 2) and the boundary conditions of Sec. 4, not from the
paper's LBM formulas, so that a mistake in the oracle's scheme shows up as a
disagreement.  Lattice units: dx = dt = 1, mu = 1.
"""
import math

import numpy as np


def couette(y, y0, y1, u0, u1):
    """Plane Couette flow between walls at y0 (velocity u0) and y1 (u1)."""
    y = np.asarray(y, dtype=np.float64)
    return u0 + (u1 - u0) * (y - y0) / (y1 - y0)


def reactive_channel_rational(y, y0, y1, D, kappa0, kappa1, K, C_top):
    """Steady C(y) of a channel with given C_top at y1 and a reacting wall at y0
    whose flux into the fluid is F(C) = (kappa0 + kappa1 C) / (1 + K C): the
    profile is linear, and the wall value C_b solves the flux balance
    D (C_top - C_b) / (y1 - y0) = -F(C_b), a quadratic once multiplied by
    (1 + K C_b); the root with 1 + K C_b > 0 nearest C_top is taken."""
    L = y1 - y0
    # D (C_top - C) (1 + K C) + L (kappa0 + kappa1 C) = 0
    a = -D * K
    b = D * K * C_top - D + L * kappa1
    c = D * C_top + L * kappa0
    roots = np.roots([a, b, c]) if a != 0 else np.array([-c / b])
    roots = np.real(roots[np.isreal(roots) & (1 + K * np.real(roots) > 0)])
    Cb = roots[np.argmin(np.abs(roots - C_top))]
    return Cb + (C_top - Cb) * (np.asarray(y, dtype=np.float64) - y0) / L


def stokes_oscillating(y, t, y0, y1, U, omega, nu, phase=0.0):
    """Stokes' second problem in a channel (Sec. 5.2, Eq. 45): the wall at y1
    moves with U cos(omega t + phase), the wall at y0 is at rest.  The periodic
    state of u_t = nu u_yy is Re[U e^{i(omega t + phase)} sinh(k (y - y0)) /
    sinh(k (y1 - y0))] with k = (1 + i) sqrt(omega / (2 nu)), the solution of
    the boundary-value problem nu w'' = i omega w, w(y0) = 0, w(y1) = U."""
    k = (1 + 1j) * np.sqrt(omega / (2 * nu))
    w = U * np.sinh(k * (np.asarray(y, dtype=np.float64) - y0)) / np.sinh(k * (y1 - y0))
    return np.real(w * np.exp(1j * (omega * t + phase)))


def poiseuille(y, y0, y1, accel, nu):
    """Body-force-driven channel flow nu u'' + a = 0, u(y0) = u(y1) = 0."""
    y = np.asarray(y, dtype=np.float64)
    return accel / (2.0 * nu) * (y - y0) * (y1 - y)


def reactive_channel(y, y0, y1, D, kappa0, kappa1, C_top):
    """Steady 1-D diffusion between a flux wall at y0 (fluid above it) with
    -D dC/dn = F(C) = kappa0 + kappa1 C (Eq. 17, n into the fluid) and a wall
    with given C = C_top at y1.  C is linear; its wall value follows from
    -D (C_top - C_b)/L = kappa0 + kappa1 C_b."""
    L = y1 - y0
    Cb = (kappa0 + D * C_top / L) / (D / L - kappa1)
    y = np.asarray(y, dtype=np.float64)
    return Cb + (C_top - Cb) * (y - y0) / L


def hartmann(y, H, B0, nu, eta, accel=0.0, rho=1.0, U_lo=0.0, U_hi=0.0,
             wall_lo=("insulating",), wall_hi=("insulating",)):
    """Steady Hartmann / Hartmann-Couette flow on -H <= y <= H.

    u = (u(y), 0), B = (b(y), B0) with mu = 1:
        nu u'' + (B0/rho) b' + accel = 0,     eta b'' + B0 u' = 0.
    Walls: u = U_lo / U_hi; b by wall type:
        ("insulating",)   b = 0
        ("conducting",)   db/dn = 0
        ("shercliff", cw) -eta db/dn = -eta b / (cw H)   (Eq. 30, n into the fluid)
    Returns (u(y), b(y)).
    Derivation: eta b' = K1 - B0 u, so u'' - M^2 u = const with M^2 =
    B0^2/(rho nu eta); u = c1 cosh(My) + c2 sinh(My) + P and
    b = -(accel rho/B0) y - (B0/(eta M)) (c1 sinh(My) + c2 cosh(My)) + K2.
    The four constants come from the four wall conditions (basis scaled by
    cosh(MH) for conditioning)."""
    M = B0 / math.sqrt(rho * nu * eta)
    ch = math.cosh(M * H)

    def basis(yy):
        # columns: c1, c2, P, K2 ; rows u, b, b'
        cy, sy = np.cosh(M * yy) / ch, np.sinh(M * yy) / ch
        u = np.stack([cy, sy, np.ones_like(yy), np.zeros_like(yy)], -1)
        b = np.stack([-(B0 / (eta * M)) * sy, -(B0 / (eta * M)) * cy, np.zeros_like(yy), np.ones_like(yy)], -1)
        db = np.stack([-(B0 / eta) * cy, -(B0 / eta) * sy, np.zeros_like(yy), np.zeros_like(yy)], -1)
        u0 = np.zeros_like(yy)
        b0 = -(accel * rho / B0) * yy
        db0 = -(accel * rho / B0) * np.ones_like(yy)
        return u, b, db, u0, b0, db0

    A = np.zeros((4, 4))
    rhs = np.zeros(4)
    for row, (yw, U, wall, nsign) in enumerate(((-H, U_lo, wall_lo, 1.0), (H, U_hi, wall_hi, -1.0))):
        u, b, db, u0, b0, db0 = basis(np.array(yw))
        A[2 * row] = u
        rhs[2 * row] = U - u0
        kind = wall[0]
        if kind == "insulating":
            A[2 * row + 1] = b
            rhs[2 * row + 1] = -b0
        elif kind == "conducting":
            A[2 * row + 1] = db
            rhs[2 * row + 1] = -db0
        elif kind == "shercliff":
            cw = wall[1]
            # d b/dn = nsign * b'; condition  d b/dn - b/(cw H) = 0
            A[2 * row + 1] = nsign * db - b / (cw * H)
            rhs[2 * row + 1] = -(nsign * db0 - b0 / (cw * H))
        else:
            raise ValueError(kind)
    c = np.linalg.solve(A, rhs)
    yy = np.asarray(y, dtype=np.float64)
    u, b, db, u0, b0, db0 = basis(yy)
    return u @ c + u0, b @ c + b0


def reaction_diffusion_series(x, y, L, W, D, k, C_bc, C_eq, nterms=400):
    """Steady diffusion on [0, L] x [0, W] (Sec. 5.3 / Fig. 6): C = C_bc at
    x = 0, dC/dx = 0 at x = L, dC/dy = 0 at y = 0, and at the reactive wall
    y = W the flux condition -D dC/dn = k (C_eq - C) with n = -y, i.e.
    D C_y + k (C - C_eq) = 0.

    Separation of variables for theta = C - C_eq:
        theta = sum_n A_n cos(l_n y) cosh(l_n (L - x)) / cosh(l_n L)
    with l_n tan(l_n W) = k/D (one root in each (n pi, n pi + pi/2)/W) and
    A_n = theta0 * int_0^W cos(l_n y) dy / int_0^W cos^2(l_n y) dy."""
    from scipy.optimize import brentq
    Bi = k / D
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    theta0 = C_bc - C_eq
    out = np.zeros(np.broadcast(x, y).shape)
    for n in range(nterms):
        lo = n * math.pi / W + 1e-14
        hi = (n * math.pi + math.pi / 2) / W - 1e-14
        lam = brentq(lambda l: l * math.tan(l * W) - Bi, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=200)
        num = math.sin(lam * W) / lam
        den = W / 2.0 + math.sin(2 * lam * W) / (4 * lam)
        An = theta0 * num / den
        # cosh(l(L-x))/cosh(lL) evaluated without overflow
        ratio = np.exp(-lam * x) * (1 + np.exp(-2 * lam * (L - x))) / (1 + math.exp(-2 * lam * L))
        out += An * np.cos(lam * y) * ratio
    return C_eq + out


def reactive_channel_two_species(y, y0, y1, DA, DB, k, A_top, B_top):
    """Steady 1-D diffusion of two species A and B between a wall at y0 where
    they react, A + B -> products at the rate k A B per unit area (each
    species' flux into the fluid is -k A B, Sec. 4.2.2), and a wall at y1 with
    given A_top, B_top.  Both profiles are linear; the wall values satisfy
    D_A (A_top - A_b) / L = D_B (B_top - B_b) / L = k A_b B_b.  Eliminating B_b
    leaves k (D_A/D_B) a^2 + (k B_top - k (D_A/D_B) A_top + D_A/L) a - D_A A_top/L
    = 0 for a = A_b, whose positive root is taken.  Returns (A(y), B(y))."""
    L = y1 - y0
    r = DA / DB
    alpha = k * r
    beta = k * B_top - k * r * A_top + DA / L
    gamma = -DA * A_top / L
    a = (-beta + math.sqrt(beta * beta - 4.0 * alpha * gamma)) / (2.0 * alpha)
    b = B_top - r * (A_top - a)
    y = np.asarray(y, dtype=np.float64)
    t = (y - y0) / L
    return a + (A_top - a) * t, b + (B_top - b) * t
