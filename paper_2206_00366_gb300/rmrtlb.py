"""Thin ctypes binding of the rmrtlb C ABI (include/rmrtlb.h).

The functions below carry the C names and only marshal arguments: every step
of the collide-and-stream path runs in the CUDA kernels of librmrtlb.so.
Pointers are plain integers (host or device addresses, e.g.
``tensor.data_ptr()`` or ``array.ctypes.data``).  A nonzero status raises
RmrtlbError.  There is no fallback: if the library is missing, loading it
raises.

``Solver`` is a convenience wrapper that takes its device workspace and its
stream from PyTorch.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "librmrtlb.so")

D2Q9, D3Q19, D3Q27, D2Q5, D3Q7 = 0, 1, 2, 3, 4
EQ_NSE, EQ_NSE_HELUO, EQ_NCDE_LINEAR, EQ_NCDE_QUAD = 0, 1, 2, 3
EQ_NCDE_SIMPLE_LINEAR, EQ_NCDE_SIMPLE_QUAD = 4, 5
BASIS_RAW, BASIS_CENTRAL, BASIS_HERMITE, BASIS_CENTRAL_HERMITE = 0, 1, 2, 3
ST_F64, ST_F32, ST_F16, ST_BF16, ST_E3M12 = 0, 1, 2, 3, 4
OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETOOBIG, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
NOALLOC_MAX_NODES = 67108864

LATTICE_NAMES = {"D2Q9": D2Q9, "D3Q19": D3Q19, "D3Q27": D3Q27, "D2Q5": D2Q5, "D3Q7": D3Q7}
STORAGE_NAMES = {"f64": ST_F64, "f32": ST_F32, "f16": ST_F16, "bf16": ST_BF16, "e3m12": ST_E3M12}
EQ_NAMES = {"nse": EQ_NSE, "nse_heluo": EQ_NSE_HELUO, "ncde_linear": EQ_NCDE_LINEAR,
            "ncde_quad": EQ_NCDE_QUAD, "ncde_simple_linear": EQ_NCDE_SIMPLE_LINEAR,
            "ncde_simple_quad": EQ_NCDE_SIMPLE_QUAD}
BASIS_NAMES = {"raw": BASIS_RAW, "central": BASIS_CENTRAL, "hermite": BASIS_HERMITE,
               "central_hermite": BASIS_CENTRAL_HERMITE}


class RmrtlbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {rmrtlb_strerror(status)} ({status})")


class rmrtlb_params(ctypes.Structure):
    _fields_ = [
        ("cs2", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("nu_bulk", ctypes.c_double),
        ("s_free", ctypes.c_double),
        ("s0", ctypes.c_double),
        ("s1", ctypes.c_double),
        ("s_shear", ctypes.c_double * 3),
        ("s_bulk", ctypes.c_double * 3),
        ("s_off", ctypes.c_double * 3),
        ("diffusivity", ctypes.c_double),
        ("adv", ctypes.c_double * 3),
        ("force", ctypes.c_double * 3),
        ("source", ctypes.c_double),
        ("check_every", ctypes.c_int),
        ("storage_range", ctypes.c_double),
        ("node_offset", ctypes.c_longlong),
    ]


class rmrtlb_domain(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("nu", ctypes.c_double), ("nu_bulk", ctypes.c_double),
        ("s_free", ctypes.c_double), ("lid_u", ctypes.c_double), ("cs2", ctypes.c_double),
    ]


def make_params(**kw) -> rmrtlb_params:
    """rmrtlb_params from keyword arguments (missing fields are zero)."""
    p = rmrtlb_params()
    for k, v in kw.items():
        if isinstance(getattr(p, k), ctypes.Array):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = float(x)
        else:
            setattr(p, k, v)
    return p


_lib = None
_vp = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load librmrtlb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(paper_2206_00366_gb300.build.build())")
    L = ctypes.CDLL(LIB_PATH)
    i, d, sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "rmrtlb_strerror": (ctypes.c_char_p, [i]),
        "rmrtlb_lattice_info": (i, [i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "rmrtlb_workspace_bytes": (i, [i, i, i, i, i, ctypes.POINTER(sz)]),
        "rmrtlb_create": (i, [ctypes.POINTER(_vp), i, i, i, i, d, d, d, d, ctypes.POINTER(rmrtlb_params),
                              i, i, i, _vp, sz, _vp]),
        "rmrtlb_destroy": (i, [_vp]),
        "rmrtlb_get_constants": (i, [_vp, ctypes.POINTER(d), i]),
        "rmrtlb_init_equilibrium": (i, [_vp, _vp, _vp]),
        "rmrtlb_set_populations": (i, [_vp, _vp]),
        "rmrtlb_get_populations": (i, [_vp, _vp]),
        "rmrtlb_step": (i, [_vp, i]),
        "rmrtlb_moments": (i, [_vp, _vp, _vp]),
        "rmrtlb_stats": (i, [_vp, ctypes.POINTER(d)]),
        "rmrtlb_last_check": (i, [_vp, ctypes.POINTER(d)]),
        "rmrtlb_check": (i, [_vp]),
        "rmrtlb_check_sums": (i, [_vp, ctypes.POINTER(d)]),
        "rmrtlb_halo_bytes": (i, [_vp, ctypes.POINTER(sz)]),
        "rmrtlb_halo_pack": (i, [_vp, _vp, _vp]),
        "rmrtlb_halo_unpack": (i, [_vp, _vp, _vp]),
        "rmrtlb_step_interior": (i, [_vp]),
        "rmrtlb_step_boundary": (i, [_vp]),
        "rmrtlb_state_bytes": (i, [_vp, ctypes.POINTER(sz)]),
        "rmrtlb_save_state": (i, [_vp, _vp, sz]),
        "rmrtlb_load_state": (i, [_vp, _vp, sz]),
        "rmrtlb_stress": (i, [_vp, _vp, _vp]),
        "rmrtlb_population_totals_noalloc": (i, [i, i, i, i, d, d, d, d, _vp, _vp, _vp]),
        "rmrtlb_batch_workspace_bytes": (i, [i, i, ctypes.POINTER(rmrtlb_domain), i, ctypes.POINTER(sz)]),
        "rmrtlb_batch_create": (i, [ctypes.POINTER(_vp), i, i, i, ctypes.POINTER(rmrtlb_domain), i, d, i, d, _vp,
                                    sz, _vp]),
        "rmrtlb_batch_run": (i, [_vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
        "rmrtlb_conv3d_forward": (i, [i, i, i, i, i, i, _vp, _vp, _vp, i, _vp, _vp, _vp]),
        "rmrtlb_conv3d_backward_data": (i, [i, i, i, i, i, i, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
        "rmrtlb_conv3d_backward_data_scratch": (ctypes.c_size_t, [i, i, i, i, i, i]),
        "rmrtlb_conv3d_backward_weight_scratch": (sz, [i, i, i, i, i, i]),
        "rmrtlb_conv3d_backward_weight": (i, [i, i, i, i, i, i, _vp, _vp, _vp, _vp, _vp, sz, _vp]),
        "rmrtlb_mse": (i, [ctypes.c_longlong, _vp, _vp, _vp, _vp, _vp, _vp]),
        "rmrtlb_adam": (i, [ctypes.c_longlong, _vp, _vp, _vp, _vp, _vp, i, ctypes.c_float, ctypes.c_float,
                            ctypes.c_float, ctypes.c_float, _vp]),
        "rmrtlb_cavity_features": (i, [i, i, i, i, _vp, _vp, _vp]),
        "rmrtlb_upsample_fields": (i, [i, i, i, i, _vp, i, i, i, ctypes.POINTER(d), ctypes.POINTER(d), _vp, _vp]),
        "rmrtlb_pack_fields": (i, [ctypes.c_longlong, i, _vp, _vp, d, d, d, _vp, _vp]),
        "rmrtlb_cnn_check": (i, [_vp]),
        "rmrtlb_cnn_wait_selftest": (i, [ctypes.c_uint, _vp]),
        "rmrtlb_batch_init_fields": (i, [_vp, i, _vp, _vp, i]),
        "rmrtlb_batch_destroy": (i, [_vp]),
        "rmrtlb_batch_reset": (i, [_vp]),
        "rmrtlb_batch_tune": (i, [_vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "rmrtlb_batch_set_launch": (i, [_vp, i, i, i]),
        "rmrtlb_batch_step": (i, [_vp, i]),
        "rmrtlb_batch_status": (i, [_vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)]),
        "rmrtlb_batch_set_populations": (i, [_vp, i, _vp]),
        "rmrtlb_batch_get_populations": (i, [_vp, i, _vp]),
        "rmrtlb_batch_fields": (i, [_vp, i, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols() -> list:
    return ["rmrtlb_strerror", "rmrtlb_lattice_info", "rmrtlb_workspace_bytes", "rmrtlb_create",
            "rmrtlb_destroy", "rmrtlb_get_constants", "rmrtlb_init_equilibrium",
            "rmrtlb_set_populations", "rmrtlb_get_populations", "rmrtlb_step", "rmrtlb_moments",
            "rmrtlb_stats", "rmrtlb_last_check", "rmrtlb_check", "rmrtlb_check_sums", "rmrtlb_halo_bytes", "rmrtlb_halo_pack",
            "rmrtlb_state_bytes", "rmrtlb_save_state", "rmrtlb_load_state", "rmrtlb_step_interior",
            "rmrtlb_step_boundary",
            "rmrtlb_halo_unpack", "rmrtlb_stress", "rmrtlb_population_totals_noalloc",
            "rmrtlb_batch_workspace_bytes", "rmrtlb_batch_create", "rmrtlb_batch_destroy", "rmrtlb_batch_reset",
            "rmrtlb_batch_tune", "rmrtlb_batch_set_launch", "rmrtlb_batch_step", "rmrtlb_batch_status", "rmrtlb_batch_set_populations",
            "rmrtlb_batch_get_populations", "rmrtlb_batch_fields", "rmrtlb_batch_run", "rmrtlb_batch_init_fields",
            "rmrtlb_conv3d_forward", "rmrtlb_conv3d_backward_data", "rmrtlb_conv3d_backward_data_scratch",
            "rmrtlb_conv3d_backward_weight_scratch",
            "rmrtlb_conv3d_backward_weight", "rmrtlb_mse", "rmrtlb_adam", "rmrtlb_cavity_features",
            "rmrtlb_upsample_fields", "rmrtlb_pack_fields", "rmrtlb_cnn_check", "rmrtlb_cnn_wait_selftest"]


def _check(status: int, where: str):
    if status != OK:
        raise RmrtlbError(status, where)


# ------------------------------------------------------------------ C names
def rmrtlb_strerror(status: int) -> str:
    return lib().rmrtlb_strerror(status).decode()


def rmrtlb_lattice_info(lattice: int):
    q, d = ctypes.c_int(), ctypes.c_int()
    e = (ctypes.c_int * 81)()
    _check(lib().rmrtlb_lattice_info(lattice, ctypes.byref(q), ctypes.byref(d), e), "rmrtlb_lattice_info")
    return q.value, d.value, np.array(e[: 3 * q.value], dtype=np.int64).reshape(q.value, 3)


def rmrtlb_workspace_bytes(lattice: int, nx: int, ny: int, nz: int, storage: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().rmrtlb_workspace_bytes(lattice, nx, ny, nz, storage, ctypes.byref(b)), "rmrtlb_workspace_bytes")
    return b.value


def rmrtlb_create(lattice, nx, ny, nz, dx, dy, dz, dt, params: rmrtlb_params, eq_kind, basis, storage,
                  workspace: int, workspace_bytes: int, stream: int):
    h = _vp()
    _check(lib().rmrtlb_create(ctypes.byref(h), lattice, nx, ny, nz, dx, dy, dz, dt, ctypes.byref(params),
                               eq_kind, basis, storage, workspace, workspace_bytes, stream), "rmrtlb_create")
    return h


def rmrtlb_destroy(h):
    _check(lib().rmrtlb_destroy(h), "rmrtlb_destroy")


def rmrtlb_get_constants(h) -> np.ndarray:
    out = (ctypes.c_double * 48)()
    _check(lib().rmrtlb_get_constants(h, out, 48), "rmrtlb_get_constants")
    return np.array(out[:])


def rmrtlb_init_equilibrium(h, rho: int, u: int):
    _check(lib().rmrtlb_init_equilibrium(h, rho, u), "rmrtlb_init_equilibrium")


def rmrtlb_set_populations(h, f: int):
    _check(lib().rmrtlb_set_populations(h, f), "rmrtlb_set_populations")


def rmrtlb_get_populations(h, f: int):
    _check(lib().rmrtlb_get_populations(h, f), "rmrtlb_get_populations")


def rmrtlb_step(h, n: int):
    _check(lib().rmrtlb_step(h, n), "rmrtlb_step")


def rmrtlb_moments(h, rho: int, u: int):
    _check(lib().rmrtlb_moments(h, rho, u), "rmrtlb_moments")


def rmrtlb_stats(h, allow_unstable: bool = False) -> np.ndarray:
    out = (ctypes.c_double * 8)()
    st = lib().rmrtlb_stats(h, out)
    if not (allow_unstable and st == EUNSTABLE):
        _check(st, "rmrtlb_stats")
    return np.array(out[:])


def rmrtlb_last_check(h, allow_unstable: bool = False) -> np.ndarray:
    out = (ctypes.c_double * 8)()
    st = lib().rmrtlb_last_check(h, out)
    if not (allow_unstable and st == EUNSTABLE):
        _check(st, "rmrtlb_last_check")
    return np.array(out[:])


def rmrtlb_step_interior(h):
    _check(lib().rmrtlb_step_interior(h), "rmrtlb_step_interior")


def rmrtlb_step_boundary(h):
    _check(lib().rmrtlb_step_boundary(h), "rmrtlb_step_boundary")


def rmrtlb_state_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(lib().rmrtlb_state_bytes(h, ctypes.byref(n)), "rmrtlb_state_bytes")
    return int(n.value)


def rmrtlb_save_state(h, dst: int, nbytes: int):
    _check(lib().rmrtlb_save_state(h, dst, nbytes), "rmrtlb_save_state")


def rmrtlb_load_state(h, src: int, nbytes: int):
    _check(lib().rmrtlb_load_state(h, src, nbytes), "rmrtlb_load_state")


def rmrtlb_check(h):
    _check(lib().rmrtlb_check(h), "rmrtlb_check")


def rmrtlb_check_sums(h) -> np.ndarray:
    out = (ctypes.c_double * 8)()
    _check(lib().rmrtlb_check_sums(h, out), "rmrtlb_check_sums")
    return np.array(out[:])


def rmrtlb_halo_bytes(h) -> int:
    b = ctypes.c_size_t()
    _check(lib().rmrtlb_halo_bytes(h, ctypes.byref(b)), "rmrtlb_halo_bytes")
    return b.value


def rmrtlb_halo_pack(h, up: int, down: int):
    _check(lib().rmrtlb_halo_pack(h, up, down), "rmrtlb_halo_pack")


def rmrtlb_halo_unpack(h, from_below: int, from_above: int):
    _check(lib().rmrtlb_halo_unpack(h, from_below, from_above), "rmrtlb_halo_unpack")


def rmrtlb_population_totals_noalloc(lattice, nx, ny, nz, dx, dy, dz, dt, f: int, out: int, stream: int):
    """Allocation-free FP64 totals of device populations (see include/rmrtlb.h)."""
    _check(lib().rmrtlb_population_totals_noalloc(lattice, nx, ny, nz, dx, dy, dz, dt, f, out, stream),
           "rmrtlb_population_totals_noalloc")


_DOMAIN_DEFAULTS = {"nz": 1, "dz": 1.0}


def _domains(domains):
    arr = (rmrtlb_domain * len(domains))()
    for k, dd in enumerate(domains):
        for f, _ in rmrtlb_domain._fields_:
            setattr(arr[k], f, dd.get(f, _DOMAIN_DEFAULTS.get(f, 0)))
    return arr


def rmrtlb_batch_workspace_bytes(lattice: int, domains, storage: int) -> int:
    arr = _domains(domains)
    b = ctypes.c_size_t()
    _check(lib().rmrtlb_batch_workspace_bytes(lattice, len(domains), arr, storage, ctypes.byref(b)),
           "rmrtlb_batch_workspace_bytes")
    return b.value


def rmrtlb_batch_create(lattice: int, basis: int, domains, storage, rho0, check_every, tol, workspace: int,
                        workspace_bytes: int, stream: int):
    arr = _domains(domains)
    h = _vp()
    _check(lib().rmrtlb_batch_create(ctypes.byref(h), lattice, basis, len(domains), arr, storage, rho0,
                                     check_every, tol, workspace, workspace_bytes, stream), "rmrtlb_batch_create")
    return h


def rmrtlb_batch_run(h, max_steps: int) -> int:
    done = ctypes.c_longlong()
    _check(lib().rmrtlb_batch_run(h, max_steps, ctypes.byref(done)), "rmrtlb_batch_run")
    return done.value


def rmrtlb_batch_init_fields(h, domain: int, rho: int, u: int, with_noneq: int):
    _check(lib().rmrtlb_batch_init_fields(h, domain, rho, u, with_noneq), "rmrtlb_batch_init_fields")


def rmrtlb_batch_destroy(h):
    _check(lib().rmrtlb_batch_destroy(h), "rmrtlb_batch_destroy")


def rmrtlb_batch_reset(h):
    _check(lib().rmrtlb_batch_reset(h), "rmrtlb_batch_reset")


def rmrtlb_batch_tune(h, steps: int):
    w, r, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().rmrtlb_batch_tune(h, steps, ctypes.byref(w), ctypes.byref(r), ctypes.byref(p)),
           "rmrtlb_batch_tune")
    return w.value, r.value, p.value


def rmrtlb_batch_set_launch(h, tile_width: int, tile_rows: int, nodes_per_thread: int):
    _check(lib().rmrtlb_batch_set_launch(h, tile_width, tile_rows, nodes_per_thread), "rmrtlb_batch_set_launch")


def rmrtlb_batch_step(h, n: int):
    _check(lib().rmrtlb_batch_step(h, n), "rmrtlb_batch_step")


def rmrtlb_batch_status(h, ndomains: int):
    res = (ctypes.c_double * ndomains)()
    conv = (ctypes.c_longlong * ndomains)()
    act = (ctypes.c_int * ndomains)()
    done = ctypes.c_longlong()
    _check(lib().rmrtlb_batch_status(h, res, conv, act, ctypes.byref(done)), "rmrtlb_batch_status")
    return np.array(res[:]), np.array(conv[:]), np.array(act[:]), done.value


def rmrtlb_batch_set_populations(h, domain: int, f: int):
    _check(lib().rmrtlb_batch_set_populations(h, domain, f), "rmrtlb_batch_set_populations")


def rmrtlb_batch_get_populations(h, domain: int, f: int):
    _check(lib().rmrtlb_batch_get_populations(h, domain, f), "rmrtlb_batch_get_populations")


def rmrtlb_batch_fields(h, domain: int, rho: int, u: int):
    _check(lib().rmrtlb_batch_fields(h, domain, rho, u), "rmrtlb_batch_fields")


def rmrtlb_stress(h, stress: int, strain: int):
    _check(lib().rmrtlb_stress(h, stress, strain), "rmrtlb_stress")


# ------------------------------------------------------------------ warm-start network (rmrtlb_cnn.h)
def rmrtlb_conv3d_forward(n, d, h, w, cin, cout, x, weight, bias, apply_silu, z, a, stream=0):
    _check(lib().rmrtlb_conv3d_forward(n, d, h, w, cin, cout, x, weight, bias, int(apply_silu), z, a, stream),
           "rmrtlb_conv3d_forward")


def rmrtlb_conv3d_backward_data_scratch(n, d, h, w, cin, cout) -> int:
    return int(lib().rmrtlb_conv3d_backward_data_scratch(n, d, h, w, cin, cout))


def rmrtlb_conv3d_backward_data(n, d, h, w, cin, cout, dy, weight, z_in, dx, scratch=None, scratch_bytes=0,
                                stream=0):
    _check(lib().rmrtlb_conv3d_backward_data(n, d, h, w, cin, cout, dy, weight, z_in, dx, scratch, scratch_bytes,
                                             stream), "rmrtlb_conv3d_backward_data")


def rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, cin, cout) -> int:
    return int(lib().rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, cin, cout))


def rmrtlb_conv3d_backward_weight(n, d, h, w, cin, cout, x, dy, dweight, dbias, scratch, scratch_bytes, stream=0):
    _check(lib().rmrtlb_conv3d_backward_weight(n, d, h, w, cin, cout, x, dy, dweight, dbias, scratch, scratch_bytes,
                                               stream), "rmrtlb_conv3d_backward_weight")


def rmrtlb_mse(count, y, t, dy, loss, scratch, stream=0):
    _check(lib().rmrtlb_mse(count, y, t, dy, loss, scratch, stream), "rmrtlb_mse")


def rmrtlb_adam(count, param, param_bf16, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
    _check(lib().rmrtlb_adam(count, param, param_bf16, grad, m, v, step, lr, beta1, beta2, eps, stream),
           "rmrtlb_adam")


def rmrtlb_cavity_features(n, d, h, w, re, x, stream=0):
    _check(lib().rmrtlb_cavity_features(n, d, h, w, re, x, stream), "rmrtlb_cavity_features")


def rmrtlb_upsample_fields(d, h, w, c, src, D, H, W, scale, offset, dst, stream=0):
    sc = (ctypes.c_double * c)(*[float(v) for v in scale])
    of = (ctypes.c_double * c)(*[float(v) for v in offset])
    _check(lib().rmrtlb_upsample_fields(d, h, w, c, src, D, H, W, sc, of, dst, stream), "rmrtlb_upsample_fields")


def rmrtlb_cnn_check(stream=0):
    _check(lib().rmrtlb_cnn_check(stream), "rmrtlb_cnn_check")


def rmrtlb_cnn_wait_selftest(polls, stream=0):
    _check(lib().rmrtlb_cnn_wait_selftest(polls, stream), "rmrtlb_cnn_wait_selftest")


def rmrtlb_pack_fields(n, d, rho, u, rho0, rho_scale, u_scale, out, stream=0):
    _check(lib().rmrtlb_pack_fields(n, d, rho, u, rho0, rho_scale, u_scale, out, stream), "rmrtlb_pack_fields")


# ------------------------------------------------------------------ convenience
def _raw_ptr(x) -> int:
    """Address of a contiguous numpy array or torch tensor of any type."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("numpy arrays must be contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return x.data_ptr()


def _ptr(x) -> int:
    """Address of a torch tensor or numpy array (must be contiguous float64)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("numpy arrays must be contiguous float64")
        return x.ctypes.data
    if not x.is_contiguous() or str(x.dtype) != "torch.float64":
        raise ValueError("tensors must be contiguous float64")
    return x.data_ptr()


class Solver:
    """One RMRT-LB solver whose workspace is a torch CUDA tensor.

    lattice, storage, eq_kind, basis: names ("D3Q19", "f32", "nse", "raw") or
    the integer codes.  shape = (nx, ny, nz); spacing = (dx, dy, dz).
    params: keyword dict for rmrtlb_params.
    """

    def __init__(self, lattice, shape, spacing, dt=1.0, params=None, eq_kind="nse", basis="raw",
                 storage="f32", device="cuda", stream=None):
        import torch
        self.lattice = LATTICE_NAMES.get(lattice, lattice)
        self.storage = STORAGE_NAMES.get(storage, storage)
        self.eq_kind = EQ_NAMES.get(eq_kind, eq_kind)
        self.basis = BASIS_NAMES.get(basis, basis)
        nx, ny, nz = (tuple(shape) + (1, 1))[:3]
        self.shape = (nx, ny, nz)
        self.q, self.d, self.e = rmrtlb_lattice_info(self.lattice)
        self.N = nx * ny * nz
        nbytes = rmrtlb_workspace_bytes(self.lattice, nx, ny, nz, self.storage)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
        sp = (tuple(spacing) + (1.0, 1.0))[:3]
        self.params = make_params(**(params or {}))
        self.h = rmrtlb_create(self.lattice, nx, ny, nz, float(sp[0]), float(sp[1]), float(sp[2]), float(dt),
                               self.params, self.eq_kind, self.basis, self.storage,
                               self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.rmrtlb_destroy(h)
            self.h = None

    def constants(self):
        return rmrtlb_get_constants(self.h)

    def init_equilibrium(self, rho, u=None):
        rmrtlb_init_equilibrium(self.h, _ptr(rho), _ptr(u))

    def set_populations(self, f):
        rmrtlb_set_populations(self.h, _ptr(f))

    def get_populations(self, out=None):
        if out is None:
            out = np.empty((self.q, self.shape[2], self.shape[1], self.shape[0]))
        rmrtlb_get_populations(self.h, _ptr(out))
        return out

    def step(self, n=1):
        rmrtlb_step(self.h, n)

    def moments(self, rho=None, u=None):
        if rho is None and u is None:
            rho = np.empty((self.shape[2], self.shape[1], self.shape[0]))
            u = np.empty((self.d, self.shape[2], self.shape[1], self.shape[0]))
        rmrtlb_moments(self.h, _ptr(rho), _ptr(u))
        return rho, u

    def stats(self, allow_unstable=False):
        return rmrtlb_stats(self.h, allow_unstable)

    def last_check(self, allow_unstable=False):
        return rmrtlb_last_check(self.h, allow_unstable)

    def save_state(self, out=None):
        """The solver's state blob (rmrtlb_save_state) in a new uint8 numpy
        array, or written into `out` (numpy array or CUDA tensor of at least
        rmrtlb_state_bytes bytes), which is returned."""
        n = rmrtlb_state_bytes(self.h)
        if out is None:
            out = np.empty(n, dtype=np.uint8)
        size = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        if size < n:
            raise ValueError(f"state needs {n} bytes, the buffer holds {size}")
        rmrtlb_save_state(self.h, _raw_ptr(out), n)
        return out

    def load_state(self, blob):
        """Restore a state saved by save_state (numpy array or CUDA tensor)."""
        nbytes = blob.nbytes if isinstance(blob, np.ndarray) else blob.numel() * blob.element_size()
        rmrtlb_load_state(self.h, _raw_ptr(blob), nbytes)

    def stress(self):
        """(stress, strain rate) as numpy arrays (d(d+1)/2, nz, ny, nx),
        components xx, yy, (zz), xy, (xz, yz); Eqs. (4-32), (4-33)."""
        import torch
        k = self.d * (self.d + 1) // 2
        shp = (k, self.shape[2], self.shape[1], self.shape[0])
        st = torch.empty(shp, dtype=torch.float64, device=self.workspace.device)
        sr = torch.empty(shp, dtype=torch.float64, device=self.workspace.device)
        rmrtlb_stress(self.h, st.data_ptr(), sr.data_ptr())
        self.stream.synchronize()
        return st.cpu().numpy(), sr.cpu().numpy()


class Batch:
    """Batched lid-driven cavities (rmrtlb_batch_*) on a torch workspace.

    domains: list of dicts with the rmrtlb_domain fields (nz, dz default to
    1).  A dedicated torch stream is used so that chunks can be captured as
    CUDA graphs (pass use_graphs=False to launch on the legacy default
    stream instead).
    """

    def __init__(self, domains, storage="f32", rho0=1.0, check_every=100, tol=1e-6, device="cuda",
                 use_graphs=True, lattice="D2Q9", basis="raw"):
        import torch
        self.domains = [dict(_DOMAIN_DEFAULTS, **d) for d in domains]
        self.lattice = LATTICE_NAMES.get(lattice, lattice)
        self.basis = BASIS_NAMES.get(basis, basis)
        self.q, self.d, _ = rmrtlb_lattice_info(self.lattice)
        self.storage = STORAGE_NAMES.get(storage, storage)
        nbytes = rmrtlb_batch_workspace_bytes(self.lattice, self.domains, self.storage)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = torch.cuda.Stream(device=self.workspace.device) if use_graphs else None
        sp = self.stream.cuda_stream if use_graphs else 0
        torch.cuda.synchronize()
        self.h = rmrtlb_batch_create(self.lattice, self.basis, self.domains, self.storage, rho0, check_every, tol,
                                     self.workspace.data_ptr(), nbytes, sp)
        self.tile_rows = 1
        self.nodes_per_thread = 0 if self.storage == STORAGE_NAMES["f32"] else 1   # 0: automatic

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.rmrtlb_batch_destroy(h)
            self.h = None

    def shape(self, domain):
        d = self.domains[domain]
        return (d["nz"], d["ny"], d["nx"])

    def reset(self):
        rmrtlb_batch_reset(self.h)

    def tune(self, steps=20):
        """Autotune the launch shape; returns the tile width (nodes); the
        rows per tile and the nodes per thread are kept in self.tile_rows
        and self.nodes_per_thread."""
        w, self.tile_rows, self.nodes_per_thread = rmrtlb_batch_tune(self.h, steps)
        return w

    def set_launch(self, tile_width, tile_rows, nodes_per_thread):
        """Set the launch shape directly (see tune); the state is kept."""
        rmrtlb_batch_set_launch(self.h, tile_width, tile_rows, nodes_per_thread)
        self.tile_rows, self.nodes_per_thread = tile_rows, nodes_per_thread

    def step(self, n=1):
        rmrtlb_batch_step(self.h, n)

    def run(self, max_steps):
        """Step until every domain has converged or gone unstable, or
        max_steps were issued; returns the steps issued."""
        return rmrtlb_batch_run(self.h, max_steps)

    def status(self):
        return rmrtlb_batch_status(self.h, len(self.domains))

    def set_populations(self, domain, f):
        rmrtlb_batch_set_populations(self.h, domain, _ptr(f))

    def get_populations(self, domain):
        out = np.empty((self.q,) + self.shape(domain))
        rmrtlb_batch_get_populations(self.h, domain, _ptr(out))
        return out

    def init_fields(self, domain, rho, u, noneq=False):
        """fbar = f^eq(rho, u) (+ f^ne with noneq); rho (nz, ny, nx), u (d, nz, ny, nx), float64
        numpy arrays or CUDA tensors."""
        rmrtlb_batch_init_fields(self.h, domain, _ptr(rho), _ptr(u), 1 if noneq else 0)

    def fields(self, domain):
        rho = np.empty(self.shape(domain))
        u = np.empty((self.d,) + self.shape(domain))
        rmrtlb_batch_fields(self.h, domain, _ptr(rho), _ptr(u))
        return rho, u
