"""FP64 CPU oracle of the coupled lattice-Boltzmann step and its wall-link
boundary schemes (Li, Chan, Feng & Wang, arXiv 2506.00907).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports it, and it imports
nothing from the product path.

Contents:
  * ``OracleSim``      -- ctypes wrapper of ``lbm_oracle.c`` (Eq. 1-6, 11-29, 34-35, 43)
  * ``LINK_DTYPE``     -- numpy record type of one wall link
  * ``links``          -- the oracle's own wall-link builder (flat and curved walls, Sec. 6)
  * ``analytic``       -- closed-form steady solutions used as pins
  * ``pipe_fd``        -- independent finite-difference solver of the MHD pipe problem
  * ``mlp``            -- FP64 reference of the warm-start network (forward, backward, Adam)

Parity status of each function is stated in its module header.
"""
import ctypes
import os

import numpy as np

from . import build as _build

LINK_DTYPE = np.dtype([
    ("node", "<i4"), ("field", "<i4"), ("dir", "<i4"), ("kind", "<i4"),
    ("d", "<f8"), ("u_wall", "<f8", (3,)), ("phi_wall", "<f8"),
    ("k0", "<f8"), ("k1", "<f8"),
])

# fields and link kinds (values are part of the link interface)
F, H, G0 = 0, 1, 2
VELOCITY, GIVEN, FLUX, NEUMANN_BFL = 0, 1, 2, 3
# variants the paper compares against (Eq. 15/16 for every d; simplified flux wall, Eq. 33)
VELOCITY_EQ15, FLUX_SIMPLIFIED = 4, 5
# open boundary of given density (pressure), Eq. 42/44; the inlet is VELOCITY with a normal u (Eq. 41/43)
PRESSURE = 6
# M-scheme flux wall of C with the reaction flux (kappa0 + kappa1 C_X) / (1 + K C_X), K = phi_wall
FLUX_RATIONAL = 7
# M-scheme flux wall of species i with k0 + k1 R_i(C_X) of the surface reaction network (several species)
REACTION = 8
MAX_SPECIES, MAX_REACT = 4, 4


def species_field(k):
    """Field code of concentration species k: 1 for species 0, 4 + k for k >= 1."""
    return H if k == 0 else 4 + k

_lib = None


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int] * 6 + [ctypes.c_double] * 3 + [dp, ctypes.c_void_p]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_links.restype = ctypes.c_int
        L.orc_set_links.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long]
        L.orc_init.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_moments.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.orc_populations.restype = ctypes.c_long
        L.orc_populations.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, ctypes.c_int]
        L.orc_steps.restype = ctypes.c_long
        L.orc_steps.argtypes = [ctypes.c_void_p]
        L.orc_set_wall_motion.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
        L.orc_set_wall_motion.restype = ctypes.c_int
        L.orc_sums.argtypes = [ctypes.c_void_p, dp]
        L.orc_feq.restype = ctypes.c_double
        L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_heq.restype = ctypes.c_double
        L.orc_heq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        L.orc_geq.restype = ctypes.c_double
        L.orc_geq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_guo.restype = ctypes.c_double
        L.orc_guo.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_eval_link.restype = ctypes.c_double
        L.orc_eval_link.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_lattice.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int), dp]
        L.orc_sizeof_link.restype = ctypes.c_int
        L.orc_set_species.restype = ctypes.c_int
        L.orc_set_species.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp]
        L.orc_set_network.restype = ctypes.c_int
        L.orc_set_network.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int), dp]
        L.orc_species.restype = ctypes.c_double
        L.orc_species.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        L.orc_network_rate.restype = ctypes.c_double
        L.orc_network_rate.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        assert L.orc_sizeof_link() == LINK_DTYPE.itemsize
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


def lattice(dim, scalar=False):
    """(e[q,3], w[q]) of D2Q9/D3Q19 (scalar=False) or D2Q5/D3Q7 (scalar=True)."""
    q = ctypes.c_int()
    e = (ctypes.c_int * 57)()
    w = (ctypes.c_double * 19)()
    lib().orc_lattice(dim, int(scalar), ctypes.byref(q), e, w)
    n = q.value
    return np.array(e[:3 * n]).reshape(n, 3), np.array(w[:n])


def opposite(e, a):
    for b in range(len(e)):
        if np.all(e[b] == -e[a]):
            return b
    raise ValueError(a)


def feq(dim, a, rho, u, B=None):
    return lib().orc_feq(dim, a, rho, _dp(_vec3(u)), _dp(_vec3(B)) if B is not None else None)


def heq(dim, a, C, u):
    return lib().orc_heq(dim, a, C, _dp(_vec3(u)))


def geq(dim, a, k, B, u):
    return lib().orc_geq(dim, a, k, _dp(_vec3(B)), _dp(_vec3(u)))


def guo(dim, a, tau, u, F):
    return lib().orc_guo(dim, a, tau, _dp(_vec3(u)), _dp(_vec3(F)))


class _LinkIn(ctypes.Structure):
    _fields_ = [("p_a_A", ctypes.c_double), ("p_ap_A", ctypes.c_double),
                ("p_ap_E", ctypes.c_double), ("phi_A", ctypes.c_double),
                ("phi_E", ctypes.c_double), ("B_A", ctypes.c_double * 3),
                ("B_E", ctypes.c_double * 3), ("u_A", ctypes.c_double * 3),
                ("u_E", ctypes.c_double * 3), ("C_A", ctypes.c_double * 4),
                ("C_E", ctypes.c_double * 4), ("nspecies", ctypes.c_int),
                ("net", ctypes.c_void_p)]


def eval_link(dim, link, p_a_A, p_ap_A, p_ap_E, phi_A=1.0, phi_E=1.0,
              B_A=(0, 0, 0), B_E=(0, 0, 0)):
    """The new unknown population of one link from explicit inputs at t."""
    rec = np.zeros(1, LINK_DTYPE)
    for k in LINK_DTYPE.names:
        if k in link:
            rec[k] = link[k]
    li = _LinkIn(p_a_A, p_ap_A, p_ap_E, phi_A, phi_E,
                 (ctypes.c_double * 3)(*B_A), (ctypes.c_double * 3)(*B_E))
    return lib().orc_eval_link(dim, rec.ctypes.data_as(ctypes.c_void_p), ctypes.byref(li))


class OracleSim:
    """One simulation domain on the CPU in FP64 (push form, Eq. 1, 3, 5).

    Node index n = x + nx*(y + ny*z); all axes wrap periodically; walls are
    solid nodes plus wall links.  ``solid`` is a uint8 array of shape
    (nz, ny, nx) (or (ny, nx) in 2D).
    """

    def __init__(self, dim, shape, solid, tau_nu, tau_D=1.0, tau_eta=1.0,
                 accel=(0.0, 0.0, 0.0), has_h=False, has_g=False, threads=1):
        nx, ny, nz = shape
        self.dim, self.nx, self.ny, self.nz = dim, nx, ny, nz
        self.N = nx * ny * nz
        self.has_h, self.has_g = has_h, has_g
        self.solid = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
        assert self.solid.size == self.N
        acc = _vec3(accel)
        self._h = lib().orc_create(dim, nx, ny, nz, int(has_h), int(has_g),
                                   tau_nu, tau_D, tau_eta, _dp(acc),
                                   self.solid.ctypes.data_as(ctypes.c_void_p))
        if not self._h:
            raise ValueError("bad oracle parameters")
        lib().orc_set_threads(self._h, threads)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_links(self, links):
        links = np.ascontiguousarray(links, dtype=LINK_DTYPE)
        rc = lib().orc_set_links(self._h, links.ctypes.data_as(ctypes.c_void_p), len(links))
        if rc != 0:
            raise ValueError("oracle rejected the link list (code %d)" % rc)

    def set_species(self, tau_D, C0):
        """Several concentration species (before the links and the initial
        state): tau_D[k] and the initial C0[k] of species k (species 0's C0 is
        init's)."""
        t = np.ascontiguousarray(tau_D, dtype=np.float64)
        c = np.ascontiguousarray(C0, dtype=np.float64)
        if len(t) != len(c) or lib().orc_set_species(self._h, len(t), _dp(t), _dp(c)) != 0:
            raise ValueError("bad species")
        self.nspecies = len(t)

    def set_network(self, reactions):
        """Surface reactions of REACTION links: a list of dicts with rate,
        order (per species, 0..2) and stoich (per species)."""
        n = len(reactions)
        rate = np.zeros(max(1, n))
        order = np.zeros(max(1, n) * MAX_SPECIES, dtype=np.int32)
        stoich = np.zeros(max(1, n) * MAX_SPECIES)
        for j, r in enumerate(reactions):
            rate[j] = r["rate"]
            for m, o in enumerate(r.get("order", ())):
                order[j * MAX_SPECIES + m] = o
            for m, v in enumerate(r.get("stoich", ())):
                stoich[j * MAX_SPECIES + m] = v
        if lib().orc_set_network(self._h, n, _dp(rate), order.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 _dp(stoich)) != 0:
            raise ValueError("bad reaction network")

    def species(self, k):
        """C[N] of species k at the current time (solid nodes 0)."""
        C = np.zeros(self.N)
        lib().orc_species(self._h, k, _dp(C))
        return C

    def network_rate(self, i, C):
        """The production rate R_i of the network at concentrations C."""
        c = np.zeros(MAX_SPECIES)
        c[:len(C)] = C
        return lib().orc_network_rate(self._h, i, _dp(c))

    def set_wall_motion(self, omega, phase=0.0):
        """Oscillating velocity walls: u_wall * cos(omega t + phase) (Eq. 45),
        t counting the steps from this call on."""
        if lib().orc_set_wall_motion(self._h, omega, phase) != 0:
            raise ValueError("wall motion needs static flux walls for h and g")

    def init(self, rho=None, u=None, C=None, B=None, rho0=1.0, C0=0.0, B0=(0.0, 0.0, 0.0)):
        def flat(a, k):
            if a is None:
                return None
            return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(self.N * k))
        self._keep = [flat(rho, 1), flat(u, 3), flat(C, 1), flat(B, 3)]
        b0 = _vec3(B0)
        lib().orc_init(self._h, *[_dp(a) for a in self._keep], rho0, C0, _dp(b0))

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    @property
    def steps(self):
        return lib().orc_steps(self._h)

    def moments(self):
        """dict of rho[N], u[N,3], C[N], B[N,3] at the current time."""
        rho = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        C = np.zeros(self.N)
        B = np.zeros(3 * self.N)
        lib().orc_moments(self._h, _dp(rho), _dp(u), _dp(C), _dp(B))
        return {"rho": rho, "u": u.reshape(self.N, 3), "C": C, "B": B.reshape(self.N, 3)}

    def populations(self, which):
        q = (9 if self.dim == 2 else 19) if which == 0 else (5 if self.dim == 2 else 7)
        cnt = q * self.N * (self.dim if which == 2 else 1)
        out = np.zeros(cnt)
        lib().orc_populations(self._h, which, _dp(out), 0)
        return out

    def set_populations(self, which, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        lib().orc_populations(self._h, which, _dp(v), 1)

    def sums(self):
        out = np.zeros(6)
        lib().orc_sums(self._h, _dp(out))
        return out
