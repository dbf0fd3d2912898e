"""ctypes binding of libpwadv.so: the C-ABI entry points under the same names.

Argument marshalling only -- every step of the stencil runs in the CUDA
library.  Importing this module loads the in-tree libpwadv.so and raises
ImportError if it is missing (there is no CPU fallback); build it with
``python -m paper_2009_12850_b300.build`` or ``__graft_entry__.build()``.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpwadv.so")

PW_OK, PW_ERR_ARG, PW_ERR_SHAPE, PW_ERR_ALIGN, PW_ERR_DTYPE = 0, -1, -2, -3, -4
PW_ERR_LID, PW_ERR_CUDA, PW_ERR_TIMEOUT, PW_ERR_NOMEM, PW_ERR_IO = -5, -6, -7, -8, -9
PW_ERR_RANGE = -10
PW_F64, PW_F32, PW_BF16, PW_BF16_OUT = 0, 1, 2, 3
PW_ALGO_AUTO, PW_ALGO_F64_NATIVE, PW_ALGO_F64_SPLIT = 0, 1, 2
PW_NOALLOC_MAX_NZ = 4096
PW_MAX_SCALARS = 16
PW_MAX_NZ = 4096


class pw_mesh_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.POINTER(ctypes.c_double)),
                ("rho_n", ctypes.POINTER(ctypes.c_double)),
                ("rho_w", ctypes.POINTER(ctypes.c_double)),
                ("rho0", ctypes.c_double), ("H_rho", ctypes.c_double),
                ("dtype", ctypes.c_int), ("algo", ctypes.c_int)]


class PWError(RuntimeError):
    def __init__(self, status, where, detail):
        super().__init__(f"{where}: {status} ({detail})")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libpwadv.so is not built ({LIB_PATH}); run paper_2009_12850_b300/build.py")

_c = ctypes.CDLL(LIB_PATH)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)

_SIGS = {
    "pw_mesh_create": ([ctypes.POINTER(pw_mesh_desc), _vp, ctypes.POINTER(_vp)], _i),
    "pw_mesh_destroy": ([_vp], None),
    "pw_mesh_layout": ([_vp, _i64p, _i64p, _i64p, _i64p], _i),
    "pw_mesh_coefficients": ([_vp, _dp, _dp], _i),
    "pw_mesh_algo": ([_vp, _ip], _i),
    "pw_mesh_device_status": ([_vp, _i, _vp, _ip], _i),
    "pw_mesh_set_tile": ([_vp, _i, _i], _i),
    "pw_selftest_timeout": ([_vp, ctypes.c_longlong, _vp], _i),
    "pw_mesh_get_tile": ([_vp, _ip, _ip], _i),
    "pw_halo_periodic": ([_vp, _vp, _vp, _vp, _vp], _i),
    "pw_halo_fold": ([_vp, _vp, _vp, _vp, _vp], _i),
    "pw_advect": ([_vp] + [_vp] * 6 + [_i, _vp], _i),
    "pw_advect_step": ([_vp] + [_vp] * 6 + [_d, _vp], _i),
    "pw_advect_scalars_step": ([_vp] * 4 + [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _vp], _i),
    "pw_advect_scalars": ([_vp] * 4 + [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _vp], _i),
    "pw_advect_tvd": ([_vp] * 4 + [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _i, _vp], _i),
    "pw_pipeline_create": ([_vp, _i, ctypes.POINTER(_vp)], _i),
    "pw_pipeline_destroy": ([_vp], None),
    "pw_pipeline_slab": ([_vp, _ip, _ip], _i),
    "pw_pipeline_sync": ([_vp], _i),
    "pw_pipeline_device_fields": ([_vp, ctypes.POINTER(_vp)], _i),
    "pw_advect_host": ([_vp] + [_vp] * 6 + [_i, _vp, _vp, _vp], _i),
    "pw_pipeline_reserve_scalars": ([_vp, _i], _i),
    "pw_advect_host_scalars": ([_vp] + [_vp] * 6 + [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _vp, _vp,
                                                       _vp], _i),
    "pw_advect_adjoint": ([_vp] + [_vp] * 9 + [_d, _i, _vp], _i),
    "pw_euler_adjoint": ([_vp] + [_vp] * 9 + [_d, _vp], _i),
    "pw_euler": ([_vp] + [_vp] * 6 + [_d, _vp], _i),
    "pw_residuals": ([_vp] + [_vp] * 6 + [_dp, _vp], _i),
    "pw_residual_ratios": ([_dp, _dp], _i),
    "pw_check_lid": ([_vp, _vp, _vp], _i),
    "pw_residuals_noalloc": ([_i, _i, _i, _i, _i, _dp, _dp] + [_vp] * 6 + [_dp, _vp], _i),
    "pw_batch_create": ([ctypes.POINTER(_vp), _i, _vp, ctypes.POINTER(_vp)], _i),
    "pw_batch_destroy": ([_vp], None),
    "pw_batch_set_fields": ([_vp] + [ctypes.POINTER(_vp)] * 6 + [_vp], _i),
    "pw_advect_batched": ([_vp, _i, _vp], _i),
    "pw_batch_halo": ([_vp, _vp], _i),
    "pw_batch_status": ([_vp, _i, _vp, _ip], _i),
    "pw_batch_set_tile": ([_vp, _i, _i, _vp], _i),
    "pw_batch_set_schedule": ([_vp, _i, _vp], _i),
    "pw_autotune": ([_vp] + [_vp] * 6 + [ctypes.c_char_p, _vp, _fp], _i),
    "pw_batch_autotune": ([_vp, ctypes.c_char_p, _vp, _fp], _i),
    "pw_status_string": ([_i], ctypes.c_char_p),
    "pw_last_error": ([], ctypes.c_char_p),
    "pw_version": ([], _i),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_c, _name)
    _f.argtypes = _args
    _f.restype = _res


def exported_symbols():
    """Names of the C-ABI entry points this binding expects the library to export."""
    return sorted(_SIGS)


def status_string(st: int) -> str:
    return _c.pw_status_string(st).decode()


def last_error() -> str:
    return _c.pw_last_error().decode()


def check(st: int, where: str):
    if st != PW_OK:
        raise PWError(st, where, f"{status_string(st)}: {last_error()}")


def _raw(name):
    return getattr(_c, name)


# Same names as the C-ABI; each raises PWError on a non-zero status.
def pw_mesh_create(desc, stream):
    out = _vp()
    check(_c.pw_mesh_create(ctypes.byref(desc), stream, ctypes.byref(out)), "pw_mesh_create")
    return out


def pw_mesh_destroy(mesh):
    _c.pw_mesh_destroy(mesh)


def pw_mesh_layout(mesh):
    a, b, c, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(_c.pw_mesh_layout(mesh, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
          "pw_mesh_layout")
    return a.value, b.value, c.value, d.value


def pw_mesh_coefficients(mesh, nz):
    buf = (ctypes.c_double * (12 * nz))()
    h = (ctypes.c_double * 2)()
    check(_c.pw_mesh_coefficients(mesh, buf, h), "pw_mesh_coefficients")
    return list(buf), (h[0], h[1])


def pw_mesh_algo(mesh):
    out = ctypes.c_int()
    check(_c.pw_mesh_algo(mesh, ctypes.byref(out)), "pw_mesh_algo")
    return out.value


def pw_mesh_device_status(mesh, clear, stream):
    st = ctypes.c_int()
    check(_c.pw_mesh_device_status(mesh, int(clear), stream, ctypes.byref(st)), "pw_mesh_device_status")
    return st.value


def pw_selftest_timeout(mesh, cycles, stream):
    check(_c.pw_selftest_timeout(mesh, int(cycles), stream), "pw_selftest_timeout")


def pw_mesh_set_tile(mesh, tile_j, tile_i):
    check(_c.pw_mesh_set_tile(mesh, int(tile_j), int(tile_i)), "pw_mesh_set_tile")


def pw_mesh_get_tile(mesh):
    a, b = ctypes.c_int(), ctypes.c_int()
    check(_c.pw_mesh_get_tile(mesh, ctypes.byref(a), ctypes.byref(b)), "pw_mesh_get_tile")
    return a.value, b.value


def pw_halo_periodic(mesh, f1, f2, f3, stream):
    check(_c.pw_halo_periodic(mesh, f1, f2, f3, stream), "pw_halo_periodic")


def pw_halo_fold(mesh, f1, f2, f3, stream):
    check(_c.pw_halo_fold(mesh, f1, f2, f3, stream), "pw_halo_fold")


def pw_advect(mesh, u, v, w, su, sv, sw, beta, stream):
    check(_c.pw_advect(mesh, u, v, w, su, sv, sw, int(beta), stream), "pw_advect")


def pw_advect_step(mesh, u, v, w, un, vn, wn, dt, stream):
    check(_c.pw_advect_step(mesh, u, v, w, un, vn, wn, float(dt), stream), "pw_advect_step")


def pw_advect_scalars(mesh, u, v, w, phi, sphi, beta, stream):
    """phi, sphi: sequences of device pointers (one per scalar)."""
    check(_c.pw_advect_scalars(mesh, u, v, w, len(phi), _ptrs(phi), _ptrs(sphi), int(beta), stream),
          "pw_advect_scalars")


def pw_advect_tvd(mesh, u, v, w, phi, sphi, dt, beta, stream):
    """phi, sphi: sequences of device pointers (one per scalar)."""
    check(_c.pw_advect_tvd(mesh, u, v, w, len(phi), _ptrs(phi), _ptrs(sphi), float(dt), int(beta), stream),
          "pw_advect_tvd")


SLAB_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_int)


def pw_pipeline_create(mesh, slab):
    out = _vp()
    check(_c.pw_pipeline_create(mesh, int(slab), ctypes.byref(out)), "pw_pipeline_create")
    return out


def pw_pipeline_destroy(p):
    _c.pw_pipeline_destroy(p)


def pw_pipeline_slab(p):
    a, b = ctypes.c_int(), ctypes.c_int()
    check(_c.pw_pipeline_slab(p, ctypes.byref(a), ctypes.byref(b)), "pw_pipeline_slab")
    return a.value, b.value


def pw_pipeline_sync(p):
    check(_c.pw_pipeline_sync(p), "pw_pipeline_sync")


def pw_pipeline_device_fields(p):
    arr = (_vp * 6)()
    check(_c.pw_pipeline_device_fields(p, arr), "pw_pipeline_device_fields")
    return [arr[q] for q in range(6)]


def pw_advect_host(p, u, v, w, su, sv, sw, beta, on_slab, user, stream):
    """on_slab: a SLAB_FN instance or None (the caller keeps it alive)."""
    fn = ctypes.cast(on_slab, _vp) if on_slab is not None else None
    check(_c.pw_advect_host(p, u, v, w, su, sv, sw, int(beta), fn, user, stream), "pw_advect_host")


def pw_advect_scalars_step(mesh, u, v, w, phi, phin, dt, stream):
    check(_c.pw_advect_scalars_step(mesh, u, v, w, len(phi), _ptrs(phi), _ptrs(phin), float(dt), stream),
          "pw_advect_scalars_step")


def pw_pipeline_reserve_scalars(p, n):
    check(_c.pw_pipeline_reserve_scalars(p, int(n)), "pw_pipeline_reserve_scalars")


def pw_advect_host_scalars(p, u, v, w, su, sv, sw, phi, sphi, beta, on_slab, user, stream):
    fn = ctypes.cast(on_slab, _vp) if on_slab is not None else None
    check(_c.pw_advect_host_scalars(p, u, v, w, su, sv, sw, len(phi), _ptrs(phi), _ptrs(sphi), int(beta), fn,
                                    user, stream), "pw_advect_host_scalars")


def pw_advect_adjoint(mesh, u, v, w, gsu, gsv, gsw, gu, gv, gw, alpha, beta, stream):
    check(_c.pw_advect_adjoint(mesh, u, v, w, gsu, gsv, gsw, gu, gv, gw, float(alpha), int(beta), stream),
          "pw_advect_adjoint")


def pw_euler_adjoint(mesh, u, v, w, gu_in, gv_in, gw_in, gu_out, gv_out, gw_out, dt, stream):
    check(_c.pw_euler_adjoint(mesh, u, v, w, gu_in, gv_in, gw_in, gu_out, gv_out, gw_out, float(dt),
                              stream), "pw_euler_adjoint")


def pw_euler(mesh, u, v, w, su, sv, sw, dt, stream):
    check(_c.pw_euler(mesh, u, v, w, su, sv, sw, float(dt), stream), "pw_euler")


def pw_residuals(mesh, u, v, w, su, sv, sw, stream):
    out = (ctypes.c_double * 12)()
    check(_c.pw_residuals(mesh, u, v, w, su, sv, sw, out, stream), "pw_residuals")
    return list(out)


def pw_residual_ratios(sums):
    a = (ctypes.c_double * 12)(*sums)
    out = (ctypes.c_double * 6)()
    check(_c.pw_residual_ratios(a, out), "pw_residual_ratios")
    return list(out)


def pw_residuals_noalloc(nx, ny, nz, nzp, dtype, w_uv, w_w, u, v, w, su, sv, sw, stream):
    """Conservation sums with no device allocation (w_uv, w_w: host sequences of nz floats)."""
    if len(w_uv) != nz or len(w_w) != nz:
        raise ValueError(f"w_uv and w_w must hold nz={nz} weights each (got {len(w_uv)}, {len(w_w)})")
    a = (ctypes.c_double * nz)(*w_uv)
    b = (ctypes.c_double * nz)(*w_w)
    out = (ctypes.c_double * 12)()
    check(_c.pw_residuals_noalloc(int(nx), int(ny), int(nz), int(nzp), int(dtype), a, b, u, v, w, su, sv, sw,
                                  out, stream), "pw_residuals_noalloc")
    return list(out)


def pw_check_lid(mesh, w, stream):
    return _c.pw_check_lid(mesh, w, stream)


def _ptrs(seq):
    arr = (_vp * len(seq))()
    for q, p in enumerate(seq):
        arr[q] = p
    return arr


def pw_batch_create(meshes, stream):
    out = _vp()
    check(_c.pw_batch_create(_ptrs(meshes), len(meshes), stream, ctypes.byref(out)), "pw_batch_create")
    return out


def pw_batch_destroy(batch):
    _c.pw_batch_destroy(batch)


def pw_batch_set_fields(batch, u, v, w, su, sv, sw, stream):
    check(_c.pw_batch_set_fields(batch, _ptrs(u), _ptrs(v), _ptrs(w), _ptrs(su), _ptrs(sv), _ptrs(sw),
                                 stream), "pw_batch_set_fields")


def pw_advect_batched(batch, beta, stream):
    check(_c.pw_advect_batched(batch, int(beta), stream), "pw_advect_batched")


def pw_batch_halo(batch, stream):
    check(_c.pw_batch_halo(batch, stream), "pw_batch_halo")


def pw_batch_set_tile(batch, threads, tile_i, stream):
    check(_c.pw_batch_set_tile(batch, int(threads), int(tile_i), stream), "pw_batch_set_tile")


def pw_batch_set_schedule(batch, persistent, stream):
    check(_c.pw_batch_set_schedule(batch, int(persistent), stream), "pw_batch_set_schedule")


def pw_batch_status(batch, clear, stream):
    st = ctypes.c_int()
    check(_c.pw_batch_status(batch, int(clear), stream, ctypes.byref(st)), "pw_batch_status")
    return st.value


def pw_autotune(mesh, u, v, w, su, sv, sw, cache_path, stream):
    ms = ctypes.c_float()
    cp = cache_path.encode() if cache_path else None
    check(_c.pw_autotune(mesh, u, v, w, su, sv, sw, cp, stream, ctypes.byref(ms)), "pw_autotune")
    return ms.value


def pw_batch_autotune(batch, cache_path, stream):
    ms = ctypes.c_float()
    cp = cache_path.encode() if cache_path else None
    check(_c.pw_batch_autotune(batch, cp, stream, ctypes.byref(ms)), "pw_batch_autotune")
    return ms.value


def pw_version():
    return _c.pw_version()
