"""The benchmark's cases on the oracle (test infrastructure only).

Builds ``OracleSim`` domains for the Hartmann channels (Sec. 5.4), the MHD
pipe (Sec. 6) and the flow + concentration channel with a reactive wall
(Sec. 5.3-style Robin flux, Eq. 17) from the shared input recipe
(``paper_2506_00907_gb300.inputs``: draws and their lattice parameters) and
the oracle's own wall-link builder (``oracle.links``).  Nothing here loads or
calls the product library.

Every one of these cases is invariant along x (periodic x, walls normal to
y, or the pipe axis along x) and starts from an x-invariant state, so its
solution is x-invariant at every step.  ``nx`` may therefore be set below the
case's own length (down to 1): the oracle then computes each x-row once, and
its values equal those of every row of the full-width domain (each node's
update is the same sequence of operations on the same values).

Parity status: the builders are pinned by ``tests/test_builders.py`` (equal
link lists to the product's builders) and the x-invariance by
``tests/test_oracle_workloads.py``.
"""
import os

import numpy as np

from . import F, H, G0, VELOCITY, GIVEN, FLUX, OracleSim
from . import links as LK


def _threads(threads):
    return threads or max(1, min(16, os.cpu_count() or 1))


def hartmann(P, nx=None, threads=None):
    """OracleSim of the Hartmann channel with lattice parameters P
    (``inputs.hartmann_params``): static no-slip walls, Shercliff B1 walls
    (M scheme, kappa1), given B2 = B0; x length nx (default the case's own).
    Returns (sim, solid)."""
    W = P["W"]
    nx = nx or P["shape"][0]
    shape = (nx, W + 2, 1)
    walls = LK.channel_y(2, nx, W + 2, 1, P["d"], P["d"])
    p = {(1, s, F): dict(kind=VELOCITY) for s in (0, 1)}
    p.update({(1, s, G0): dict(kind=FLUX, kappa1=P["kappa1"]) for s in (0, 1)})
    p.update({(1, s, G0 + 1): dict(kind=GIVEN, phi_wall=P["B0"]) for s in (0, 1)})
    solid = LK.box_solid(shape, walls)
    sim = OracleSim(2, shape, solid, P["tau_nu"], 1.0, P["tau_eta"], (P["accel"], 0.0, 0.0), False, True,
                    _threads(threads))
    sim.set_links(LK.box_links(2, shape, walls, p, has_g=True))
    sim.init(rho0=1.0, B0=(0.0, P["B0"], 0.0))
    return sim, solid


def pipe(P, shape, nx=None, threads=None):
    """OracleSim of the MHD pipe with lattice parameters P (``inputs.pipe_params``)
    on the grid ``shape`` (axis along x), x length nx (default shape[0]).
    B1 insulating (given 0), conducting (zero flux) or Shercliff (kappa1);
    B2 = B0 and B3 = 0 given.  Returns (sim, solid)."""
    shape = (nx or shape[0], shape[1], shape[2])
    wall = P["wall"]
    g0 = dict(kind=GIVEN, phi_wall=0.0) if wall == "insulating" else \
        dict(kind=FLUX) if wall == "conducting" else dict(kind=FLUX, kappa1=P["kappa1"])
    params = {F: dict(kind=VELOCITY), G0: g0, G0 + 1: dict(kind=GIVEN, phi_wall=P["B0"]),
              G0 + 2: dict(kind=GIVEN, phi_wall=0.0)}
    solid = LK.pipe_solid(shape, P["R"])
    links, _ = LK.pipe_links(shape, P["R"], params)
    sim = OracleSim(3, shape, solid, P["tau_nu"], 1.0, P["tau_eta"], (P["accel"], 0.0, 0.0), False, True,
                    _threads(threads))
    sim.set_links(links)
    sim.init(rho0=1.0, B0=(0.0, P["B0"], 0.0))
    return sim, solid


def reactive(P, nx=None, threads=None):
    """OracleSim of the flow + concentration channel with parameters P
    (``inputs.reactive_params``): bottom wall static with the Robin flux
    kappa0 + kappa1 C (M scheme), top wall moving at U with given C_top; C
    starts at C_eq.  Returns (sim, solid)."""
    nx = nx or P["shape"][0]
    ny = P["shape"][1]
    shape = (nx, ny, 1)
    walls = LK.channel_y(2, nx, ny, 1, P["d"], P["d"])
    U = (P["U"], 0.0, 0.0)
    p = {(1, 0, F): dict(kind=VELOCITY), (1, 1, F): dict(kind=VELOCITY, u_wall=U),
         (1, 0, H): dict(kind=FLUX, kappa0=P["kappa0"], kappa1=P["kappa1"]),
         (1, 1, H): dict(kind=GIVEN, phi_wall=P["C_top"], u_wall=U)}
    solid = LK.box_solid(shape, walls)
    sim = OracleSim(2, shape, solid, P["tau_nu"], P["tau_D"], 1.0, (0.0, 0.0, 0.0), True, False, _threads(threads))
    sim.set_links(LK.box_links(2, shape, walls, p, has_h=True))
    sim.init(rho0=1.0, C0=P["C_eq"])
    return sim, solid


def widen(field, nx):
    """Values of an x-invariant field computed on a domain of x length 1,
    repeated to x length nx (node order n = x + nx (y + ny z))."""
    return np.repeat(np.asarray(field), nx, axis=0)
