"""Shared test helpers (no method arithmetic)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def affine_fixed_point(step, q, shape, reach=1):
    """Fixed point of an affine map p -> M p + c on SoA populations (q, N).

    The map is one oracle time step with frozen velocity (pure diffusion): it is
    affine in the populations, and an output at node x depends only on inputs
    within ``reach`` nodes of x along every axis.  M is assembled exactly by
    probing all nodes of one colour (period 2*reach+1 per axis) at once, then
    (I - M) p = c is solved directly.  Returns the fixed point."""
    nx, ny, nz = shape
    N = nx * ny * nz
    n = q * N
    c = step(np.zeros(n))
    P = 2 * reach + 1
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    colour = (x % P) + P * ((y % P) + P * (z % P))
    rows, cols, vals = [], [], []

    def nearest(o, c0, n_):
        d = (c0 - o) % P
        d = np.where(d > reach, d - P, d)
        return (o + d) % n_

    for col in np.unique(colour):
        cx, cy, cz = col % P, (col // P) % P, col // (P * P)
        sel = np.flatnonzero(colour == col)
        for a in range(q):
            e = np.zeros(n)
            e[a * N + sel] = 1.0
            r = step(e) - c
            nzr = np.flatnonzero(r)
            if nzr.size == 0:
                continue
            on = nzr % N
            sx = nearest(x[on], cx, nx)
            sy = nearest(y[on], cy, ny)
            sz = nearest(z[on], cz, nz)
            rows.append(nzr)
            cols.append(a * N + sx + nx * (sy + ny * sz))
            vals.append(r[nzr])
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return spla.spsolve((sp.identity(n, format="csr") - M).tocsc(), c)


def norm_rel(a, b):
    """max|a - b| / max|b| (per-field norm-relative difference)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def to_abi_links(orc_links):
    """Copy oracle link records field by field into the C-ABI record layout."""
    from paper_2506_00907_gb300 import lbm
    out = np.zeros(len(orc_links), dtype=lbm.LINK_DTYPE)
    for k in ("node", "field", "dir", "kind", "d", "u_wall", "phi_wall", "k0", "k1"):
        out[k] = orc_links[k]
    return out


def sort_links(links):
    order = np.lexsort((links["dir"], links["field"], links["node"]))
    return links[order]
