"""Independent finite-volume solver of the steady MHD pipe problem (Sec. 6),
used to pin the oracle's curved-wall results (test infrastructure only).

Fully developed flow along the pipe axis x1 with B_ext = (0, B0, 0) along x2
(mu = 1):
    nu lap u + (B0/rho) db/dx2 + a = 0,     eta lap b + B0 du/dx2 = 0
on the disk r < R, with u = 0 at r = R and, for the induced axial field b:
    insulating  b = 0;  conducting  db/dr = 0 (b then fixed to zero area mean);
    Shercliff   -eta db/dn = -eta b/(cw R), n = -r (into the fluid),
                i.e. db/dr + b/(cw R) = 0   (Eq. 30 with H = R, Sec. 6.2).
Discretisation: cell-centred polar grid r_i = (i + 1/2) dr, theta_j = j dtheta;
conservative second-order Laplacian (the flux through r = 0 vanishes);
central differences for d/dx2 = cos(t) d/dr - sin(t)/r d/dt, the value across
the centre taken from the opposite ray; wall conditions through one ghost ring.
The solution is second order in dr and dtheta.  This solver shares nothing
with the lattice-Boltzmann code.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def solve(R, B0, nu, eta, accel, rho=1.0, wall=("insulating",), nr=96, nt=192, src=None):
    """Returns (r[nr], theta[nt], u[nr, nt], b[nr, nt]).

    ``src(y, z) -> (su, sb)`` optionally adds source terms to the right-hand
    sides of the two equations (used by manufactured-solution tests)."""
    assert nt % 2 == 0
    dr = R / nr
    dt = 2.0 * np.pi / nt
    r = (np.arange(nr) + 0.5) * dr
    th = np.arange(nt) * dt
    kind = wall[0]
    if kind == "insulating":
        gb = -1.0
    elif kind == "conducting":
        gb = 1.0
    elif kind == "shercliff":
        beta = dr / (2.0 * wall[1] * R)
        gb = (1.0 - beta) / (1.0 + beta)
    else:
        raise ValueError(kind)
    gu = -1.0   # u = 0 at r = R
    n = nr * nt

    def idx(i, j):
        return i * nt + (j % nt)

    rows, cols, vals = [], [], []

    def add(row, col, v):
        rows.append(row)
        cols.append(col)
        vals.append(v)

    rhs = np.zeros(2 * n)
    for i in range(nr):
        ri = r[i]
        rp = ri + 0.5 * dr
        rm = ri - 0.5 * dr
        for j in range(nt):
            c, s = np.cos(th[j]), np.sin(th[j])
            p = idx(i, j)
            for field in (0, 1):            # 0: u-equation, 1: b-equation
                row = field * n + p
                lam, g_self = (nu, gu) if field == 0 else (eta, gb)
                # Laplacian of the own variable
                own = field * n
                diag = -(rp + (rm if i > 0 else 0.0)) / (ri * dr * dr) - 2.0 / (ri * ri * dt * dt)
                if i + 1 < nr:
                    add(row, own + idx(i + 1, j), lam * rp / (ri * dr * dr))
                else:
                    diag += g_self * rp / (ri * dr * dr)
                if i > 0:
                    add(row, own + idx(i - 1, j), lam * rm / (ri * dr * dr))
                add(row, own + idx(i, j + 1), lam / (ri * ri * dt * dt))
                add(row, own + idx(i, j - 1), lam / (ri * ri * dt * dt))
                add(row, own + p, lam * diag)
                # d/dx2 of the other variable, times the coupling
                oth = (1 - field) * n
                coup = B0 / rho if field == 0 else B0
                g_oth = gb if field == 0 else gu
                # radial derivative
                if i + 1 < nr:
                    add(row, oth + idx(i + 1, j), coup * c / (2 * dr))
                else:
                    add(row, oth + p, coup * c * g_oth / (2 * dr))
                if i > 0:
                    add(row, oth + idx(i - 1, j), -coup * c / (2 * dr))
                else:
                    add(row, oth + idx(0, j + nt // 2), -coup * c / (2 * dr))
                # azimuthal derivative
                add(row, oth + idx(i, j + 1), -coup * s / (ri * 2 * dt))
                add(row, oth + idx(i, j - 1), coup * s / (ri * 2 * dt))
            rhs[p] = -accel
            if src is not None:
                su, sb = src(ri * c, ri * s)
                rhs[p] -= su
                rhs[n + p] -= sb
    if kind != "conducting":
        A = sp.csc_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n))
        x = spla.spsolve(A, rhs)
    else:
        # db/dn = 0 fixes b only up to a constant: border the system with the
        # zero area-mean condition on b (one Lagrange multiplier).
        wts = np.repeat(r, nt)
        for p in range(n):
            add(2 * n, n + p, wts[p])
            add(n + p, 2 * n, wts[p])
        A = sp.csc_matrix((vals, (rows, cols)), shape=(2 * n + 1, 2 * n + 1))
        x = spla.spsolve(A, np.concatenate([rhs, [0.0]]))
    return r, th, x[:n].reshape(nr, nt), x[n:2 * n].reshape(nr, nt)


def sample(r, th, field, yy, zz):
    """Bilinear interpolation of a polar field at Cartesian points (y, z)
    relative to the axis (periodic in theta, linear in r, extrapolated to the
    wall)."""
    rr = np.hypot(yy, zz)
    tt = np.mod(np.arctan2(zz, yy), 2 * np.pi)
    nr, nt = field.shape
    dr = r[1] - r[0]
    dt = th[1] - th[0]
    fi = np.clip(rr / dr - 0.5, 0.0, nr - 1.0)
    i0 = np.clip(np.floor(fi).astype(int), 0, nr - 2)
    wi = fi - i0
    fj = tt / dt
    j0 = np.floor(fj).astype(int) % nt
    wj = fj - np.floor(fj)
    j1 = (j0 + 1) % nt
    v = ((1 - wi) * (1 - wj) * field[i0, j0] + wi * (1 - wj) * field[i0 + 1, j0]
         + (1 - wi) * wj * field[i0, j1] + wi * wj * field[i0 + 1, j1])
    # near the wall (beyond the last cell centre) extrapolate linearly in r
    out = rr > r[-1]
    if np.any(out):
        w = (rr[out] - r[-1]) / dr
        ja, jb, wjo = j0[out], j1[out], wj[out]
        last = (1 - wjo) * field[nr - 1, ja] + wjo * field[nr - 1, jb]
        prev = (1 - wjo) * field[nr - 2, ja] + wjo * field[nr - 2, jb]
        v[out] = last + w * (last - prev)
    return v


def mean_velocity(r, th, u):
    """Area average of u over the disk (midpoint rule on the polar cells)."""
    dr = r[1] - r[0]
    dt = th[1] - th[0]
    area = np.sum(r) * dr * dt * len(th)
    return np.sum(u * r[:, None]) * dr * dt / area
