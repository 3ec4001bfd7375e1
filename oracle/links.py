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

from . import (LINK_DTYPE, F, H, G0, VELOCITY, GIVEN, FLUX, NEUMANN_BFL, VELOCITY_EQ15, FLUX_SIMPLIFIED,
               FLUX_RATIONAL, REACTION, lattice, species_field)


def _fields(dim, has_h, has_g, nspecies=1):
    out = [F]
    if has_h:
        out += [species_field(k) for k in range(nspecies)]
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


def _records(nodes, field, a, kind, d, u_wall, phi_wall, k0, k1):
    r = np.zeros(len(nodes), LINK_DTYPE)
    r["node"], r["field"], r["dir"], r["kind"], r["d"] = nodes, field, a, kind, d
    r["u_wall"] = np.broadcast_to(np.asarray(u_wall, dtype=np.float64), (len(nodes), 3)) if len(nodes) else 0
    r["phi_wall"], r["k0"], r["k1"] = phi_wall, k0, k1
    return r


def _upstream_solid(solid3, e):
    """mask over nodes A of solid[A - e] (periodic)."""
    return np.roll(solid3, shift=(e[2], e[1], e[0]), axis=(0, 1, 2))


def box_links(dim, shape, walls, params, has_h=False, has_g=False, nspecies=1):
    """Links of a box with planar walls.

    walls:  axis -> (lo, hi) wall coordinates (see ``box_solid``).
    params: (axis, side, field) -> dict(kind, u_wall, phi_wall, kappa0, kappa1)
            with side 0 = lo wall, 1 = hi wall.
    d is the distance along the link to the first wall plane it crosses
    (s in (0, 1] with A - s e_a on the plane); ties at corners go to the wall
    listed first in ``walls`` (lo before hi).
    """
    nx, ny, nz = shape
    solid3 = box_solid(shape, walls)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = (x.ravel(), y.ravel(), z.ravel())
    out = []
    for field in _fields(dim, has_h, has_g, nspecies):
        e, _ = lattice(dim, scalar=(field != F))
        for a in range(1, len(e)):
            mask = (solid3 == 0) & (_upstream_solid(solid3, e[a]) == 1)
            nodes = np.flatnonzero(mask.ravel())
            if nodes.size == 0:
                continue
            best = np.full(nodes.size, np.inf)
            which = np.full(nodes.size, -1)
            cands = []
            for ax, (lo, hi) in walls.items():
                if e[a][ax] == 0:
                    continue
                for side, pos in ((0, lo), (1, hi)):
                    cands.append((ax, side, pos))
            for ci, (ax, side, pos) in enumerate(cands):
                s = (coords[ax][nodes] - pos) / e[a][ax]
                ok = (s > 0.0) & (s <= 1.0 + 1e-12) & (s < best - 1e-12)
                best = np.where(ok, np.minimum(s, 1.0), best)
                which = np.where(ok, ci, which)
            if np.any(which < 0):
                raise ValueError("a fluid node next to a solid node has no wall between them")
            for ci, (ax, side, pos) in enumerate(cands):
                sel = which == ci
                if not np.any(sel):
                    continue
                p = params[(ax, side, field)]
                out.append(_records(nodes[sel], field, a, p["kind"], best[sel], p.get("u_wall", (0, 0, 0)),
                                    p.get("phi_wall", 0.0), p.get("kappa0", 0.0), p.get("kappa1", 0.0)))
    if not out:
        return np.zeros(0, LINK_DTYPE)
    return np.concatenate(out)


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
    return (ae + np.sqrt(disc)) / ee


def pipe_segments(shape, R, center=None):
    """Outer-layer solid points of every axial slice with their surface element
    S_i = (theta_{i+1} - theta_{i-1}) R / 2 (dx = 1) and inward normal.

    Returns dict node -> (S_i, n_i[3])."""
    nx, ny, nz = shape
    cy, cz = center if center is not None else ((ny - 1) / 2.0, (nz - 1) / 2.0)
    solid3 = pipe_solid(shape, R, center)
    e7, _ = lattice(3, scalar=True)
    touches = np.zeros_like(solid3, dtype=bool)
    for g in range(1, 7):
        # neighbour B + e_g is fluid
        touches |= np.roll(solid3, shift=(-e7[g][2], -e7[g][1], -e7[g][0]), axis=(0, 1, 2)) == 0
    outer = (solid3 == 1) & touches
    out = {}
    for x in range(nx):
        zz, yy = np.nonzero(outer[:, :, x])
        nodes = x + nx * (yy + ny * zz)
        th = np.arctan2(zz - cz, yy - cy)
        order = np.lexsort((nodes, th))
        th, nodes, yy, zz = th[order], nodes[order], yy[order], zz[order]
        th_next = np.roll(th, -1)
        th_next[-1] += 2 * np.pi
        th_prev = np.roll(th, 1)
        th_prev[0] -= 2 * np.pi
        S = (th_next - th_prev) * R / 2.0
        r = np.hypot(yy - cy, zz - cz)
        for i in range(len(nodes)):
            out[int(nodes[i])] = (float(S[i]), np.array([0.0, -(yy[i] - cy) / r[i], -(zz[i] - cz) / r[i]]))
    return out


def pipe_links(shape, R, params, has_g=True, center=None):
    """Links of the pipe (flow D3Q19 + vector B on D3Q7).

    params: field -> dict(kind, u_wall, phi_wall, kappa0, kappa1).
    Flux coefficients are multiplied by S_B and the split weight of Eq. 48.
    Returns (links, info) with info = dict(segments, e_solid_links).
    """
    nx, ny, nz = shape
    cy, cz = center if center is not None else ((ny - 1) / 2.0, (nz - 1) / 2.0)
    solid3 = pipe_solid(shape, R, center)
    solid = solid3.reshape(-1)
    segs = pipe_segments(shape, R, center)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    out = []
    e_solid = 0
    e7, _ = lattice(3, scalar=True)
    for field in _fields(3, False, has_g):
        e, _ = lattice(3, scalar=(field != F))
        p = params[field]
        for a in range(1, len(e)):
            mask = ((solid3 == 0) & (_upstream_solid(solid3, e[a]) == 1)).ravel()
            nodes = np.flatnonzero(mask)
            if nodes.size == 0:
                continue
            d = ray_circle_d(y[nodes] - cy, z[nodes] - cz, e[a][1], e[a][2], R)
            d = np.minimum(np.maximum(d, 1e-12), 1.0)
            En = (x[nodes] + e[a][0]) % nx + nx * (((y[nodes] + e[a][1]) % ny) + ny * ((z[nodes] + e[a][2]) % nz))
            e_solid += int(np.sum(solid[En]))
            k0 = np.zeros(nodes.size)
            k1 = np.zeros(nodes.size)
            if p["kind"] in (FLUX, FLUX_SIMPLIFIED, FLUX_RATIONAL):
                bx, by, bz = (x[nodes] - e[a][0]) % nx, (y[nodes] - e[a][1]) % ny, (z[nodes] - e[a][2]) % nz
                Bn = bx + nx * (by + ny * bz)
                for i in range(nodes.size):
                    S, nB = segs[int(Bn[i])]
                    tot = 0.0
                    for g in range(1, 7):
                        pg = float(np.dot(e7[g], nB))
                        Ag = (bx[i] + e7[g][0]) % nx + nx * (((by[i] + e7[g][1]) % ny) + ny * ((bz[i] + e7[g][2]) % nz))
                        if pg > 0 and not solid[Ag]:
                            tot += pg
                    ea_n = float(np.dot(e[a], nB))
                    w = ea_n / tot if ea_n > 0 else 0.0
                    k0[i] = p.get("kappa0", 0.0) * S * w
                    k1[i] = p.get("kappa1", 0.0) * S * w
            out.append(_records(nodes, field, a, p["kind"], d, p.get("u_wall", (0, 0, 0)),
                                p.get("phi_wall", 0.0), k0, k1))
    return np.concatenate(out), {"segments": segs, "e_solid_links": e_solid}


# ---------------------------------------------------------------------------
# Random links for parity fuzzing
# ---------------------------------------------------------------------------
def random_links(dim, shape, solid, rng, has_h=False, has_g=False, kinds=None, phi_range=None, variants=False,
                 nspecies=1, reaction=False):
    """Every required link of a given solid mask, with kind, d and wall data
    drawn from ``rng`` (numpy Generator).  d in (0, 1]; both branches of every
    scheme occur.  phi_range maps a field to the (lo, hi) range of its given
    wall values (default (-0.5, 1.5)).  variants=True also draws the two
    comparison schemes (Eq. 15/16 for every d, the simplified flux wall).
    nspecies concentration fields; reaction=True also draws reaction links
    (k1 in (0.5, 1], the area weight of the network's rate)."""
    nx, ny, nz = shape
    solid3 = np.asarray(solid, dtype=np.uint8).reshape(nz, ny, nx)
    out = []
    for field in _fields(dim, has_h, has_g, nspecies):
        e, _ = lattice(dim, scalar=(field != F))
        is_c = field == H or field >= G0 + 3
        if field == F:
            allowed = np.array([VELOCITY, VELOCITY_EQ15] if variants else [VELOCITY])
        else:
            allowed = np.array(kinds or ([GIVEN, FLUX, NEUMANN_BFL, FLUX_SIMPLIFIED] if variants
                                         else [GIVEN, FLUX, NEUMANN_BFL]))
            if reaction and is_c:
                allowed = np.concatenate([allowed, [REACTION, REACTION]])
        for a in range(1, len(e)):
            nodes = np.flatnonzero(((solid3 == 0) & (_upstream_solid(solid3, e[a]) == 1)).ravel())
            m = nodes.size
            if m == 0:
                continue
            r = np.zeros(m, LINK_DTYPE)
            r["node"], r["field"], r["dir"] = nodes, field, a
            r["kind"] = allowed[rng.integers(len(allowed), size=m)]
            r["d"] = 1.0 - rng.random(m)
            uw = rng.uniform(-0.02, 0.02, (m, 3))
            if dim == 2:
                uw[:, 2] = 0.0
            r["u_wall"] = uw
            lo, hi = (phi_range or {}).get(field, (-0.5, 1.5))
            r["phi_wall"] = rng.uniform(lo, hi, m)
            r["k0"] = rng.uniform(-0.01, 0.01, m)
            r["k1"] = rng.uniform(-0.05, 0.0, m)
            react = r["kind"] == REACTION
            r["k1"][react] = rng.uniform(0.5, 1.0, int(react.sum()))
            out.append(r)
    if not out:
        return np.zeros(0, LINK_DTYPE)
    return np.concatenate(out)
