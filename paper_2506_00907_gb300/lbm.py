"""Thin ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every function named ``lbm_*`` here calls the C entry point of the same name in
``liblbm_gb300.so``; all arithmetic runs in the CUDA kernels.  ``Solver`` is a
small convenience wrapper over those calls.  There is no CPU fallback: if the
library cannot be built or loaded, or no GPU is present, calls raise.
"""
import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE = range(7)
LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_FP64, LBM_FP32, LBM_FP16S, LBM_BF16S = 0, 1, 2, 3
LBM_FLOW, LBM_CD, LBM_MHD = 1, 2, 4
LBM_W_VELOCITY, LBM_W_GIVEN, LBM_W_FLUX, LBM_W_NEUMANN_BFL = 0, 1, 2, 3
LBM_W_VELOCITY_EQ15, LBM_W_FLUX_SIMPLIFIED = 4, 5      # the paper's comparison schemes
LBM_W_PRESSURE = 6                                      # open boundary of given density (Eq. 42, 44)
LBM_W_REACTION = 8                                      # surface reaction network, several species (Sec. 4.2.2)
FIELD_F, FIELD_H, FIELD_G = 0, 1, 2
LBM_MAX_SPECIES, LBM_MAX_REACT = 3, 4


def field_species(k):
    """Field code of concentration species k (LBM_FIELD_SPECIES)."""
    return 1 if k == 0 else 4 + k
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16s": LBM_FP16S, "bf16s": LBM_BF16S}

LINK_DTYPE = np.dtype([
    ("node", "<u4"), ("field", "u1"), ("dir", "u1"), ("kind", "u1"), ("reserved", "u1"),
    ("d", "<f8"), ("u_wall", "<f8", (3,)), ("phi_wall", "<f8"), ("k0", "<f8"), ("k1", "<f8"),
])
assert LINK_DTYPE.itemsize == 64


class lbm_case(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("tau_nu", ctypes.c_double), ("tau_D", ctypes.c_double), ("tau_eta", ctypes.c_double),
                ("accel", ctypes.c_double * 3), ("rho0", ctypes.c_double), ("C0", ctypes.c_double),
                ("B0", ctypes.c_double * 3), ("tau_Dk", ctypes.c_double * 3), ("C0k", ctypes.c_double * 3)]


class lbm_config(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("prec", ctypes.c_int), ("physics", ctypes.c_uint32),
                ("ncases", ctypes.c_int32), ("cases", ctypes.POINTER(lbm_case)),
                ("stream", ctypes.c_void_p), ("device", ctypes.c_int32), ("nspecies", ctypes.c_int32)]


class lbm_reaction(ctypes.Structure):
    _fields_ = [("rate", ctypes.c_double), ("order", ctypes.c_int32 * 3), ("stoich", ctypes.c_double * 3)]


class lbm_launch(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("nodes_per_thread", ctypes.c_int32), ("stages", ctypes.c_int32), ("min_blocks", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lbm status %d: %s" % (status, msg))
        self.status = status


_LIB = None


def lib():
    """Load liblbm_gb300.so (building it first if it is missing)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            path = _build.build()
        L = ctypes.CDLL(path)
        vp, i32, i64, dp, fp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, \
            ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
        sig = {
            "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_config), ctypes.POINTER(vp)]),
            "lbm_destroy": (None, [vp]),
            "lbm_last_error": (ctypes.c_char_p, [vp]),
            "lbm_set_walls": (ctypes.c_int, [vp, i32, vp, vp, ctypes.c_size_t]),
            "lbm_init_equilibrium": (ctypes.c_int, [vp, i32, dp, dp, dp, dp]),
            "lbm_init_equilibrium_device": (ctypes.c_int, [vp, i32, fp, fp, fp, fp]),
            "lbm_step": (ctypes.c_int, [vp, i32]),
            "lbm_set_graph": (ctypes.c_int, [vp, i32]),
            "lbm_set_wall_motion": (ctypes.c_int, [vp, i32, ctypes.c_double, ctypes.c_double]),
            "lbm_moments": (ctypes.c_int, [vp, i32, dp, dp, dp, dp]),
            "lbm_check": (ctypes.c_int, [vp, dp]),
            "lbm_check_async": (ctypes.c_int, [vp]),
            "lbm_check_wait": (ctypes.c_int, [vp, dp]),
            "lbm_run_to_steady": (ctypes.c_int, [vp, i64, i32, ctypes.c_double,
                                                 ctypes.POINTER(i64), dp]),
            "lbm_set_active": (ctypes.c_int, [vp, i32, i32]),
            "lbm_run_each_to_steady": (ctypes.c_int, [vp, i64, i32, ctypes.c_double,
                                                      ctypes.POINTER(i64), dp]),
            "lbm_state_bytes": (ctypes.c_size_t, [vp]),
            "lbm_get_state": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
            "lbm_set_state": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
            "lbm_steps_done": (i64, [vp]),
            "lbm_set_launch": (ctypes.c_int, [vp, ctypes.POINTER(lbm_launch)]),
            "lbm_get_launch": (ctypes.c_int, [vp, ctypes.POINTER(lbm_launch)]),
            "lbm_autotune": (ctypes.c_int, [vp, ctypes.c_char_p, i32, ctypes.POINTER(lbm_launch), dp]),
            "lbm_launches_per_step": (i32, [vp]),
            "lbm_device_state": (ctypes.c_int, [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(i32),
                                                ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)]),
        }
        sig["lbm_build_channel"] = (ctypes.c_int, [i32, i32, i32, i32, i32, ctypes.c_double, ctypes.c_double,
                                                    ctypes.c_uint32, vp, vp, vp, ctypes.c_size_t,
                                                    ctypes.POINTER(ctypes.c_size_t)])
        sig["lbm_build_pipe"] = (ctypes.c_int, [i32, i32, i32, ctypes.c_double, ctypes.c_uint32, vp, vp, vp,
                                                ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)])
        sig["lbm_convert_state"] = (ctypes.c_int, [vp, vp])
        sig["lbm_net_num_params"] = (i64, [])
        sig["lbm_net_create"] = (ctypes.c_int, [ctypes.POINTER(i32), i32, vp, vp, ctypes.POINTER(vp)])
        sig["lbm_net_destroy"] = (None, [vp])
        sig["lbm_net_get_params"] = (ctypes.c_int, [vp, vp])
        sig["lbm_net_set_params"] = (ctypes.c_int, [vp, vp])
        sig["lbm_net_forward"] = (ctypes.c_int, [vp, vp, vp, i64])
        sig["lbm_net_loss_grad"] = (ctypes.c_int, [vp, vp, vp, i64, dp, vp])
        sig["lbm_net_adam"] = (ctypes.c_int, [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float])
        sig["lbm_net_pipe_fields"] = (ctypes.c_int, [vp, i32, i32, i32, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_double, vp, vp])
        sig["lbm_reduce_noalloc"] = (ctypes.c_int, [i32, i32, ctypes.c_uint32, ctypes.POINTER(lbm_case), vp, i64,
                                                     vp, vp, dp, vp])
        sig["lbm_species"] = (ctypes.c_int, [vp, i32, i32, dp])
        sig["lbm_set_reactions"] = (ctypes.c_int, [vp, i32, i32, ctypes.POINTER(lbm_reaction)])
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(ctx, st):
    if st != LBM_OK:
        raise LbmError(st, lib().lbm_last_error(ctx).decode())


# ----------------------------------------------------------------- C-ABI mirrors
def lbm_create(lattice, prec, physics, cases, stream=None, device=0, nspecies=0):
    arr = (lbm_case * len(cases))(*cases)
    cfg = lbm_config(lattice, prec, physics, len(cases), arr, stream, device, nspecies)
    h = ctypes.c_void_p()
    _check(None, lib().lbm_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def lbm_destroy(ctx):
    lib().lbm_destroy(ctx)


def lbm_set_walls(ctx, case_id, solid, links):
    solid = np.ascontiguousarray(np.asarray(solid).reshape(-1).astype(np.uint8))
    links = np.ascontiguousarray(links, dtype=LINK_DTYPE)
    _check(ctx, lib().lbm_set_walls(ctx, case_id, solid.ctypes.data, links.ctypes.data if len(links) else None,
                                    len(links)))


def lbm_init_equilibrium(ctx, case_id, rho=None, u=None, C=None, B=None):
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (rho, u, C, B)]
    _check(ctx, lib().lbm_init_equilibrium(ctx, case_id, *[_dp(a) for a in arrs]))


def lbm_init_equilibrium_device(ctx, case_id, rho=None, u=None, C=None, B=None):
    """Fields are device pointers (int) or torch float32 CUDA tensors."""
    def ptr(t):
        if t is None:
            return None
        return t if isinstance(t, int) else t.data_ptr()
    _check(ctx, lib().lbm_init_equilibrium_device(ctx, case_id, ptr(rho), ptr(u), ptr(C), ptr(B)))


def lbm_step(ctx, nsteps):
    _check(ctx, lib().lbm_step(ctx, int(nsteps)))


def lbm_set_graph(ctx, steps_per_graph):
    _check(ctx, lib().lbm_set_graph(ctx, int(steps_per_graph)))


def lbm_set_wall_motion(ctx, case_id, omega, phase=0.0):
    _check(ctx, lib().lbm_set_wall_motion(ctx, int(case_id), float(omega), float(phase)))


def lbm_moments(ctx, case_id, N):
    rho, u, C, B = np.zeros(N), np.zeros(3 * N), np.zeros(N), np.zeros(3 * N)
    _check(ctx, lib().lbm_moments(ctx, case_id, _dp(rho), _dp(u), _dp(C), _dp(B)))
    return {"rho": rho, "u": u.reshape(N, 3), "C": C, "B": B.reshape(N, 3)}


def lbm_species(ctx, case_id, k, N):
    C = np.zeros(N)
    _check(ctx, lib().lbm_species(ctx, case_id, k, _dp(C)))
    return C


def lbm_set_reactions(ctx, case_id, reactions):
    """reactions: list of dicts with rate, order (per species, 0..2) and stoich (per species)."""
    n = len(reactions)
    arr = (lbm_reaction * max(1, n))()
    for j, r in enumerate(reactions):
        arr[j].rate = r["rate"]
        for m, o in enumerate(r.get("order", ())):
            arr[j].order[m] = int(o)
        for m, v in enumerate(r.get("stoich", ())):
            arr[j].stoich[m] = float(v)
    _check(ctx, lib().lbm_set_reactions(ctx, case_id, n, arr))


def lbm_check(ctx, ncases, raise_unstable=True):
    out = np.zeros(8 * ncases)
    st = lib().lbm_check(ctx, _dp(out))
    if st != LBM_OK and (st != LBM_EUNSTABLE or raise_unstable):
        _check(ctx, st)
    return out.reshape(ncases, 8)


def lbm_check_async(ctx):
    _check(ctx, lib().lbm_check_async(ctx))


def lbm_check_wait(ctx, ncases, raise_unstable=True):
    out = np.zeros(8 * ncases)
    st = lib().lbm_check_wait(ctx, _dp(out))
    if st != LBM_OK and (st != LBM_EUNSTABLE or raise_unstable):
        _check(ctx, st)
    return out.reshape(ncases, 8)


def lbm_run_to_steady(ctx, max_steps, interval, tol):
    done = ctypes.c_int64()
    res = ctypes.c_double()
    _check(ctx, lib().lbm_run_to_steady(ctx, int(max_steps), int(interval), float(tol),
                                        ctypes.byref(done), ctypes.byref(res)))
    return done.value, res.value


def lbm_set_active(ctx, case_id, active):
    _check(ctx, lib().lbm_set_active(ctx, int(case_id), 1 if active else 0))


def lbm_run_each_to_steady(ctx, max_steps, interval, tol):
    done = ctypes.c_int64()
    res = ctypes.c_double()
    _check(ctx, lib().lbm_run_each_to_steady(ctx, int(max_steps), int(interval), float(tol),
                                             ctypes.byref(done), ctypes.byref(res)))
    return done.value, res.value


def lbm_get_state(ctx):
    n = lib().lbm_state_bytes(ctx)
    buf = np.zeros(n, dtype=np.uint8)
    _check(ctx, lib().lbm_get_state(ctx, buf.ctypes.data, n))
    return buf


def lbm_set_state(ctx, blob):
    blob = np.ascontiguousarray(blob, dtype=np.uint8)
    _check(ctx, lib().lbm_set_state(ctx, blob.ctypes.data, blob.size))


def lbm_steps_done(ctx):
    return lib().lbm_steps_done(ctx)


def launch(variant=0, block=256, blocks_per_sm=0, nodes_per_thread=1, stages=2, min_blocks=1):
    return lbm_launch(variant, block, blocks_per_sm, nodes_per_thread, stages, min_blocks)


def lbm_set_launch(ctx, lp):
    _check(ctx, lib().lbm_set_launch(ctx, ctypes.byref(lp)))


def lbm_get_launch(ctx):
    lp = lbm_launch()
    _check(ctx, lib().lbm_get_launch(ctx, ctypes.byref(lp)))
    return lp


def lbm_autotune(ctx, cache_path=None, iters=20):
    lp, ms = lbm_launch(), ctypes.c_double()
    _check(ctx, lib().lbm_autotune(ctx, cache_path.encode() if cache_path else None, int(iters), ctypes.byref(lp),
                                   ctypes.byref(ms)))
    return lp, ms.value


def lbm_reduce_noalloc(lattice, prec, physics, case, pops, plane_stride, flags=None, snap=None, stream=None):
    """Allocation-free FP64 reduction of one domain's stored populations (see
    include/lbm.h): pops, flags and snap are device pointers (ints) the caller
    owns; returns the 8-number record of lbm_check."""
    out = np.zeros(8)
    st = lib().lbm_reduce_noalloc(lattice, prec, physics, ctypes.byref(case), pops, int(plane_stride), flags, snap,
                                  _dp(out), stream)
    if st not in (LBM_OK, LBM_EUNSTABLE):
        raise LbmError(st, "lbm_reduce_noalloc failed")
    return out, st


def lbm_convert_state(dst, src):
    """Copy the state of context `src` into `dst` at the precision of `dst`."""
    _check(dst, lib().lbm_convert_state(dst, src))


def lbm_launches_per_step(ctx):
    return lib().lbm_launches_per_step(ctx)


def lbm_device_state(ctx, case_id):
    base, eb, ps, off, planes = ctypes.c_void_p(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64(), \
        ctypes.c_int32()
    _check(ctx, lib().lbm_device_state(ctx, case_id, ctypes.byref(base), ctypes.byref(eb), ctypes.byref(ps),
                                       ctypes.byref(off), ctypes.byref(planes)))
    return dict(base=base.value, elem_bytes=eb.value, plane_stride=ps.value, case_offset=off.value,
                planes=planes.value)


class lbm_wall_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("u_wall", ctypes.c_double * 3), ("phi_wall", ctypes.c_double),
                ("kappa0", ctypes.c_double), ("kappa1", ctypes.c_double)]


def wall_bc(kind=LBM_W_VELOCITY, u_wall=(0.0, 0.0, 0.0), phi_wall=0.0, kappa0=0.0, kappa1=0.0):
    return lbm_wall_bc(kind, (ctypes.c_double * 3)(*u_wall), phi_wall, kappa0, kappa1)


def _bc_array(bcs, n):
    arr = (lbm_wall_bc * n)()
    for i, b in enumerate(bcs):
        if b is not None:
            arr[i] = b
    return arr


def lbm_build_channel(dim, shape, axis, d_lo, d_hi, physics, bc_lo, bc_hi):
    """bc_lo / bc_hi: 5 lbm_wall_bc (fields f, h, g_0, g_1, g_2; None = unused).
    Returns (solid uint8[N], links LINK_DTYPE)."""
    nx, ny, nz = shape
    bcs = _bc_array(list(bc_lo) + list(bc_hi), 10)
    solid = np.zeros(nx * ny * nz, dtype=np.uint8)
    cnt = ctypes.c_size_t()
    st = lib().lbm_build_channel(dim, nx, ny, nz, axis, d_lo, d_hi, physics, bcs, solid.ctypes.data, None, 0,
                                 ctypes.byref(cnt))
    if st != LBM_OK:
        raise LbmError(st, "lbm_build_channel: bad arguments")
    links = np.zeros(cnt.value, dtype=LINK_DTYPE)
    st = lib().lbm_build_channel(dim, nx, ny, nz, axis, d_lo, d_hi, physics, bcs, solid.ctypes.data,
                                 links.ctypes.data, cnt.value, ctypes.byref(cnt))
    if st != LBM_OK:
        raise LbmError(st, "lbm_build_channel failed")
    return solid, links


def lbm_build_pipe(shape, R, physics, bcs):
    """bcs: 5 lbm_wall_bc (fields f, h, g_0, g_1, g_2).  Returns (solid, links)."""
    nx, ny, nz = shape
    arr = _bc_array(bcs, 5)
    solid = np.zeros(nx * ny * nz, dtype=np.uint8)
    cnt = ctypes.c_size_t()
    st = lib().lbm_build_pipe(nx, ny, nz, R, physics, arr, solid.ctypes.data, None, 0, ctypes.byref(cnt))
    if st != LBM_OK:
        raise LbmError(st, "lbm_build_pipe: bad arguments")
    links = np.zeros(cnt.value, dtype=LINK_DTYPE)
    st = lib().lbm_build_pipe(nx, ny, nz, R, physics, arr, solid.ctypes.data, links.ctypes.data, cnt.value,
                              ctypes.byref(cnt))
    if st != LBM_OK:
        raise LbmError(st, "lbm_build_pipe failed")
    return solid, links


NET_DIMS = (4, 64, 64, 64, 2)


def _st(st, what):
    if st != LBM_OK:
        raise LbmError(st, what)


class Net:
    """The warm-start network (include/lbm.h, lbm_net_*): device parameters,
    the library's forward / backward / Adam kernels."""

    def __init__(self, init_params, stream=None):
        init = np.ascontiguousarray(init_params, dtype=np.float32)
        assert init.size == lib().lbm_net_num_params()
        dims = (ctypes.c_int32 * 5)(*NET_DIMS)
        h = ctypes.c_void_p()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        _st(lib().lbm_net_create(dims, 5, init.ctypes.data, stream, ctypes.byref(h)), "lbm_net_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def num_params():
        return lib().lbm_net_num_params()

    def get_params(self):
        out = np.zeros(self.num_params(), dtype=np.float32)
        _st(lib().lbm_net_get_params(self.h, out.ctypes.data), "lbm_net_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _st(lib().lbm_net_set_params(self.h, p.ctypes.data), "lbm_net_set_params")

    def forward(self, x, y):
        """x, y: torch float32 CUDA tensors [n, 4] and [n, 2]."""
        _st(lib().lbm_net_forward(self.h, x.data_ptr(), y.data_ptr(), x.shape[0]), "lbm_net_forward")

    def loss_grad(self, x, t, want_grad=False):
        loss = ctypes.c_double()
        g = np.zeros(self.num_params(), dtype=np.float32) if want_grad else None
        _st(lib().lbm_net_loss_grad(self.h, x.data_ptr(), t.data_ptr(), x.shape[0], ctypes.byref(loss),
                                    g.ctypes.data if want_grad else None), "lbm_net_loss_grad")
        return loss.value, g

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _st(lib().lbm_net_adam(self.h, lr, beta1, beta2, eps), "lbm_net_adam")

    def pipe_fields(self, shape, R, f_ha, f_cw, u_scale, b_scale, B0, u, B):
        nx, ny, nz = shape
        _st(lib().lbm_net_pipe_fields(self.h, nx, ny, nz, R, f_ha, f_cw, u_scale, b_scale, B0, u.data_ptr(),
                                      B.data_ptr()), "lbm_net_pipe_fields")


# ----------------------------------------------------------------- convenience
def make_case(shape, tau_nu, tau_D=1.0, tau_eta=1.0, accel=(0.0, 0.0, 0.0), rho0=1.0, C0=0.0,
              B0=(0.0, 0.0, 0.0), tau_Dk=(1.0, 1.0, 1.0), C0k=(0.0, 0.0, 0.0)):
    """tau_Dk, C0k: relaxation times and initial C of concentration species 1..3."""
    nx, ny, nz = shape
    td = list(tau_Dk) + [1.0] * (3 - len(tau_Dk))
    c0 = list(C0k) + [0.0] * (3 - len(C0k))
    return lbm_case(nx, ny, nz, tau_nu, tau_D, tau_eta, (ctypes.c_double * 3)(*accel), rho0, C0,
                    (ctypes.c_double * 3)(*B0), (ctypes.c_double * 3)(*td), (ctypes.c_double * 3)(*c0))


class Solver:
    """One context: all cases share lattice, precision and physics and are
    advanced together, one fused launch per step."""

    def __init__(self, lattice, prec, physics, cases, stream=None, device=0, nspecies=0):
        if isinstance(prec, str):
            prec = PRECISIONS[prec]
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.cases = list(cases)
        self.N = [c.nx * c.ny * c.nz for c in self.cases]
        self.lattice, self.prec, self.physics = lattice, prec, physics
        self.ctx = lbm_create(lattice, prec, physics, self.cases, stream, device, nspecies)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_walls(self, case_id, solid, links):
        lbm_set_walls(self.ctx, case_id, solid, links)

    def init_equilibrium(self, case_id, **fields):
        lbm_init_equilibrium(self.ctx, case_id, **fields)

    def init_equilibrium_device(self, case_id, **fields):
        lbm_init_equilibrium_device(self.ctx, case_id, **fields)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def set_graph(self, k):
        lbm_set_graph(self.ctx, k)

    def set_wall_motion(self, case_id, omega, phase=0.0):
        lbm_set_wall_motion(self.ctx, case_id, omega, phase)

    def moments(self, case_id=0):
        return lbm_moments(self.ctx, case_id, self.N[case_id])

    def species(self, k, case_id=0):
        """Concentration of species k (N entries)."""
        return lbm_species(self.ctx, case_id, k, self.N[case_id])

    def set_reactions(self, case_id, reactions):
        lbm_set_reactions(self.ctx, case_id, reactions)

    def check(self, raise_unstable=True):
        return lbm_check(self.ctx, len(self.cases), raise_unstable)

    def check_async(self):
        lbm_check_async(self.ctx)

    def check_wait(self, raise_unstable=True):
        return lbm_check_wait(self.ctx, len(self.cases), raise_unstable)

    def run_to_steady(self, max_steps, interval=100, tol=1e-8):
        return lbm_run_to_steady(self.ctx, max_steps, interval, tol)

    def set_active(self, case_id, active):
        """Freeze (False) or resume (True) one case; see lbm_set_active."""
        lbm_set_active(self.ctx, case_id, active)

    def run_each_to_steady(self, max_steps, interval=500, tol=1e-9):
        """Freeze each case once its own residual is below tol; returns
        (time steps of the batch, largest last residual)."""
        return lbm_run_each_to_steady(self.ctx, max_steps, interval, tol)

    def get_state(self):
        return lbm_get_state(self.ctx)

    def set_state(self, blob):
        lbm_set_state(self.ctx, blob)

    def convert_from(self, other):
        """Take the state of Solver `other` (same cases and walls), rounded to this precision."""
        lbm_convert_state(self.ctx, other.ctx)

    @property
    def steps(self):
        return lbm_steps_done(self.ctx)

    def set_launch(self, variant=0, block=256, blocks_per_sm=0, nodes_per_thread=1, stages=2, min_blocks=1):
        lbm_set_launch(self.ctx, launch(variant, block, blocks_per_sm, nodes_per_thread, stages, min_blocks))

    def get_launch(self):
        return lbm_get_launch(self.ctx).as_dict()

    def autotune(self, cache_path=None, iters=20):
        return lbm_autotune(self.ctx, cache_path, iters)
