"""Oracle wall-link builder (test infrastructure only).

Builds the list of wall links (A, field, a, kind, d, wall data) from a
geometry, written independently of the product's builder:

* Flat walls (boxes / channels): the wall is a plane; d = AX/|EA| is the same
  for axis and diagonal directions (Sec. 4.1, remark after Eq. 16).
* Curved pipe wall (Sec. 6): d per node and per direction from the ray-circle
  intersection (Fig. 9a); surface segmentation S_i = (theta_{i+1} -
  theta_{i-1}) R dx / 2 over the outer-layer solid points sorted by azimuth;
  conservative flux splitting over the links of each solid point (Eq. 48).

Conventions: node n = x + nx*(y + ny*z); every axis wraps; a link exists for
every fluid node A, field and direction a with B = A - e_a solid; a is the
unknown direction at A (pointing from the wall into the fluid).
For flux links the stored coefficients are per step and per link:
k0 = kappa0 * S_B * w_a and k1 = kappa1 * S_B * w_a, where the wall flux is
F(phi) = kappa0 + kappa1 * phi (lattice units, Eq. 23), S_B = 1 for flat walls.
"""
import math

import numpy as np

from . import LINK_DTYPE, F, H, G0, VELOCITY, GIVEN, FLUX, NEUMANN_BFL, lattice


def _fields(dim, has_h, has_g):
    out = [F]
    if has_h:
        out.append(H)
    if has_g:
        out += [G0 + k for k in range(dim)]
    return out


def _wrap(v, n):
    return v % n


def box_solid(shape, walls):
    """uint8 solid mask (nz, ny, nx) of a box whose bounded axes carry planar
    walls.  ``walls`` maps axis -> (lo, hi) wall coordinates; node i is fluid
    along that axis iff lo < i < hi.  Unlisted axes are periodic."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = (x, y, z)
    fluid = np.ones((nz, ny, nx), dtype=bool)
    for ax, (lo, hi) in walls.items():
        c = coords[ax]
        fluid &= (c > lo) & (c < hi)
    return (~fluid).astype(np.uint8)


def _link_record(node, field, a, kind, d, u_wall=(0, 0, 0), phi_wall=0.0, k0=0.0, k1=0.0):
    r = np.zeros(1, LINK_DTYPE)
    r["node"], r["field"], r["dir"], r["kind"], r["d"] = node, field, a, kind, d
    r["u_wall"] = u_wall
    r["phi_wall"], r["k0"], r["k1"] = phi_wall, k0, k1
    return r


def box_links(dim, shape, walls, params, has_h=False, has_g=False):
    """Links of a box with planar walls.

    walls:  axis -> (lo, hi) wall coordinates (see ``box_solid``).
    params: (axis, side, field) -> dict(kind, u_wall, phi_wall, kappa0, kappa1)
            with side 0 = lo wall, 1 = hi wall.
    Ties at corners (two walls crossed at the same distance) go to the wall
    listed first in ``walls`` (lo before hi).
    """
    nx, ny, nz = shape
    solid = box_solid(shape, walls).reshape(-1)
    recs = []
    for field in _fields(dim, has_h, has_g):
        e, _ = lattice(dim, scalar=(field != F))
        for n in np.flatnonzero(solid == 0):
            x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
            A = (x, y, z)
            for a in range(1, len(e)):
                bx, by, bz = _wrap(x - e[a][0], nx), _wrap(y - e[a][1], ny), _wrap(z - e[a][2], nz)
                if not solid[bx + nx * (by + ny * bz)]:
                    continue
                # first wall crossed by the ray A - s e_a, s in (0, 1]
                best = None
                for ax, (lo, hi) in walls.items():
                    if e[a][ax] == 0:
                        continue
                    for side, pos in ((0, lo), (1, hi)):
                        s = (A[ax] - pos) / e[a][ax]
                        if 0.0 < s <= 1.0 + 1e-12 and (best is None or s < best[0] - 1e-12):
                            best = (min(s, 1.0), ax, side)
                if best is None:
                    raise ValueError("no wall between fluid node %s and solid node" % (A,))
                d, ax, side = best
                p = params[(ax, side, field)]
                kind = p["kind"]
                k0 = p.get("kappa0", 0.0)
                k1 = p.get("kappa1", 0.0)
                recs.append(_link_record(n, field, a, kind, d, p.get("u_wall", (0, 0, 0)),
                                         p.get("phi_wall", 0.0), k0, k1))
    if not recs:
        return np.zeros(0, LINK_DTYPE)
    return np.concatenate(recs)


def channel_y(dim, nx, ny, nz, d_lo, d_hi):
    """Walls normal to y at y = 1 - d_lo and y = ny - 2 + d_lo (solid rows 0 and ny-1)."""
    return {1: (1.0 - d_lo, ny - 2.0 + d_hi)}


# ---------------------------------------------------------------------------
# Curved pipe wall (Sec. 6)
# ---------------------------------------------------------------------------
def pipe_solid(shape, R, center=None):
    """Axis along x; fluid iff (y-cy)^2 + (z-cz)^2 < R^2."""
    nx, ny, nz = shape
    cy, cz = center if center is not None else ((ny - 1) / 2.0, (nz - 1) / 2.0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    fluid = (y - cy) ** 2 + (z - cz) ** 2 < R * R
    return (~fluid).astype(np.uint8)


def ray_circle_d(ay, az, ey, ez, R):
    """Smallest s > 0 with |a - s e| = R for |a| < R (a relative to the centre):
    the fraction d of the link A -> B = A - e cut off by the wall (Fig. 9a)."""
    ee = ey * ey + ez * ez
    ae = ay * ey + az * ez
    disc = ae * ae + ee * (R * R - (ay * ay + az * az))
    return (ae + math.sqrt(disc)) / ee


def pipe_segments(shape, R, center=None):
    """Outer-layer solid points of every axial slice with their surface element
    S_i = (theta_{i+1} - theta_{i-1}) R / 2 (dx = 1) and inward normal.

    Returns dict node -> (S_i, n_i[3])."""
    nx, ny, nz = shape
    cy, cz = center if center is not None else ((ny - 1) / 2.0, (nz - 1) / 2.0)
    solid = pipe_solid(shape, R, center).reshape(-1)
    e7, _ = lattice(3, scalar=True)
    out = {}
    for x in range(nx):
        pts = []
        for z in range(nz):
            for y in range(ny):
                n = x + nx * (y + ny * z)
                if not solid[n]:
                    continue
                touches = False
                for g in range(1, 7):
                    A = _wrap(x + e7[g][0], nx) + nx * (_wrap(y + e7[g][1], ny) + ny * _wrap(z + e7[g][2], nz))
                    if not solid[A]:
                        touches = True
                if touches:
                    pts.append((math.atan2(z - cz, y - cy), n, y - cy, z - cz))
        pts.sort()
        m = len(pts)
        for i, (th, n, by, bz) in enumerate(pts):
            th_next = pts[(i + 1) % m][0] + (2 * math.pi if i + 1 == m else 0.0)
            th_prev = pts[(i - 1) % m][0] - (2 * math.pi if i == 0 else 0.0)
            S = (th_next - th_prev) * R / 2.0
            r = math.hypot(by, bz)
            out[n] = (S, np.array([0.0, -by / r, -bz / r]))
    return out


def pipe_links(shape, R, params, has_g=True, center=None):
    """Links of the pipe (flow D3Q19 + vector B on D3Q7).

    params: field -> dict(kind, u_wall, phi_wall, kappa0, kappa1).
    Flux coefficients are multiplied by S_B and the split weight of Eq. 48.
    Returns (links, info) with info = dict(segments, e_solid_links).
    """
    nx, ny, nz = shape
    cy, cz = center if center is not None else ((ny - 1) / 2.0, (nz - 1) / 2.0)
    solid = pipe_solid(shape, R, center).reshape(-1)
    segs = pipe_segments(shape, R, center)
    recs = []
    e_solid = 0
    for field in _fields(3, False, has_g):
        e, _ = lattice(3, scalar=(field != F))
        p = params[field]
        for n in np.flatnonzero(solid == 0):
            x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
            for a in range(1, len(e)):
                bx, by, bz = _wrap(x - e[a][0], nx), _wrap(y - e[a][1], ny), _wrap(z - e[a][2], nz)
                Bn = bx + nx * (by + ny * bz)
                if not solid[Bn]:
                    continue
                d = ray_circle_d(y - cy, z - cz, e[a][1], e[a][2], R)
                d = min(max(d, 1e-12), 1.0)
                En = _wrap(x + e[a][0], nx) + nx * (_wrap(y + e[a][1], ny) + ny * _wrap(z + e[a][2], nz))
                if solid[En]:
                    e_solid += 1
                k0 = k1 = 0.0
                if p["kind"] == FLUX:
                    S, nB = segs[Bn]
                    proj = [float(np.dot(e[g], nB)) for g in range(1, len(e))]
                    tot = 0.0
                    for g in range(1, len(e)):
                        Ag = _wrap(bx + e[g][0], nx) + nx * (_wrap(by + e[g][1], ny) + ny * _wrap(bz + e[g][2], nz))
                        if not solid[Ag] and proj[g - 1] > 0:
                            tot += proj[g - 1]
                    ea_n = float(np.dot(e[a], nB))
                    w = ea_n / tot if ea_n > 0 else 0.0
                    k0 = p.get("kappa0", 0.0) * S * w
                    k1 = p.get("kappa1", 0.0) * S * w
                recs.append(_link_record(n, field, a, p["kind"], d, p.get("u_wall", (0, 0, 0)),
                                         p.get("phi_wall", 0.0), k0, k1))
    return np.concatenate(recs), {"segments": segs, "e_solid_links": e_solid}


# ---------------------------------------------------------------------------
# Random links for parity fuzzing
# ---------------------------------------------------------------------------
def random_links(dim, shape, solid, rng, has_h=False, has_g=False, kinds=None):
    """Every required link of a given solid mask, with kind, d and wall data
    drawn from ``rng`` (numpy Generator).  d in (0, 1]; both branches of every
    scheme occur."""
    nx, ny, nz = shape
    solid = np.asarray(solid, dtype=np.uint8).reshape(-1)
    recs = []
    for field in _fields(dim, has_h, has_g):
        e, _ = lattice(dim, scalar=(field != F))
        allowed = [VELOCITY] if field == F else (kinds or [GIVEN, FLUX, NEUMANN_BFL])
        for n in np.flatnonzero(solid == 0):
            x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
            for a in range(1, len(e)):
                bx, by, bz = _wrap(x - e[a][0], nx), _wrap(y - e[a][1], ny), _wrap(z - e[a][2], nz)
                if not solid[bx + nx * (by + ny * bz)]:
                    continue
                kind = allowed[rng.integers(len(allowed))]
                d = 1.0 - rng.random()            # (0, 1]
                uw = rng.uniform(-0.02, 0.02, 3)
                if dim == 2:
                    uw[2] = 0.0
                recs.append(_link_record(n, field, a, kind, d, uw, rng.uniform(-0.5, 1.5),
                                         rng.uniform(-0.01, 0.01), rng.uniform(-0.05, 0.0)))
    if not recs:
        return np.zeros(0, LINK_DTYPE)
    return np.concatenate(recs)
