"""Torch-facing wrapper of the C-ABI: a Mesh owns a pw_mesh and allocates,
validates and passes device tensors.  PyTorch only provides device memory and
the current stream; all arithmetic happens in libpwadv.so.

Field tensors have the library layout: shape (nx+4, ny+4, nzp), contiguous,
k fastest, 2-wide periodic halos in x and y.  ``Mesh.interior(t)`` is the
(nx, ny, nz) view of the interior.
"""
import ctypes

import numpy as np
import torch

from . import _lib as L

_DT = {"f64": L.PW_F64, "f32": L.PW_F32, "bf16": L.PW_BF16, "bf16_out": L.PW_BF16_OUT}
_ALGO = {"auto": L.PW_ALGO_AUTO, "native": L.PW_ALGO_F64_NATIVE, "split": L.PW_ALGO_F64_SPLIT}
_TORCH_IN = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16, "bf16_out": torch.bfloat16}
_TORCH_OUT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.float32, "bf16_out": torch.bfloat16}


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _host(a):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Mesh:
    def __init__(self, nx, ny, nz, dx, dy=None, dz=None, rho_n=None, rho_w=None, rho0=0.0, H=0.0,
                 dtype="f64", algo="auto", device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2009_12850_b300 needs a CUDA device")
        self.device = torch.device(device or "cuda")
        self.dtype = dtype
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx = float(dx)
        self.dy = float(dx if dy is None else dy)
        self._keep = [_host(dz), _host(rho_n), _host(rho_w)]
        d = L.pw_mesh_desc()
        d.nx, d.ny, d.nz, d.dx, d.dy = self.nx, self.ny, self.nz, self.dx, self.dy
        d.dz, d.rho_n, d.rho_w = (k[1] for k in self._keep)
        d.rho0, d.H_rho = float(rho0), float(H)
        d.dtype, d.algo = _DT[dtype], _ALGO[algo]
        with torch.cuda.device(self.device):
            self.handle = L.pw_mesh_create(d, _stream())
        self.nzp, self.stride_j, self.stride_i, self.total = L.pw_mesh_layout(self.handle)
        self.in_dtype = _TORCH_IN[dtype]
        self.out_dtype = _TORCH_OUT[dtype]

    def close(self):
        if getattr(self, "handle", None):
            L.pw_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ layout
    @property
    def shape(self):
        return (self.nx + 4, self.ny + 4, self.nzp)

    def empty(self, dtype=None):
        return torch.empty(self.shape, dtype=dtype or self.in_dtype, device=self.device)

    def zeros(self, dtype=None):
        return torch.zeros(self.shape, dtype=dtype or self.in_dtype, device=self.device)

    def empty_out(self):
        return self.empty(self.out_dtype)

    def interior(self, t):
        return t[2:self.nx + 2, 2:self.ny + 2, :self.nz]

    def from_interior(self, arr, dtype=None, fill_halo=True):
        """Field tensor from an (nx, ny, nz) array: interior copied, padding 0,
        halos filled on the device by the library."""
        t = self.zeros(dtype)
        src = torch.as_tensor(np.ascontiguousarray(arr)) if isinstance(arr, np.ndarray) else arr
        self.interior(t).copy_(src.to(device=self.device, dtype=t.dtype))
        if fill_halo:
            self.halo(t)
        return t

    def _check(self, t, name, out=False):
        want = self.out_dtype if out else self.in_dtype
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != want:
            raise TypeError(f"{name} must be {want}, got {t.dtype}")
        if t.numel() != self.total or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with {self.total} elements (shape {self.shape})")
        return ctypes.c_void_p(t.data_ptr())

    # ------------------------------------------------------------------ calls
    def coefficients(self):
        vals, (tcx, tcy) = L.pw_mesh_coefficients(self.handle, self.nz)
        a = np.array(vals).reshape(12, self.nz)
        names = ["dz", "zf", "zn", "dzn", "rho_n", "rho_w", "tzc1", "tzc2", "tzd1", "tzd2", "W_uv", "W_w"]
        out = {n: a[q] for q, n in enumerate(names)}
        out["tcx"], out["tcy"] = tcx, tcy
        return out

    def halo(self, f1, f2=None, f3=None, stream=None):
        ps = [self._check(f1, "f1")] + [self._check(f, "f") if f is not None else None for f in (f2, f3)]
        L.pw_halo_periodic(self.handle, ps[0], ps[1], ps[2], _stream(stream))

    def halo_fold(self, f1, f2=None, f3=None, stream=None):
        ps = [self._check(f1, "f1")] + [self._check(f, "f") if f is not None else None for f in (f2, f3)]
        L.pw_halo_fold(self.handle, ps[0], ps[1], ps[2], _stream(stream))

    def advect(self, u, v, w, su=None, sv=None, sw=None, beta=0, stream=None):
        su = self.empty_out() if su is None else su
        sv = self.empty_out() if sv is None else sv
        sw = self.empty_out() if sw is None else sw
        L.pw_advect(self.handle, self._check(u, "u"), self._check(v, "v"), self._check(w, "w"),
                    self._check(su, "su", True), self._check(sv, "sv", True), self._check(sw, "sw", True),
                    beta, _stream(stream))
        return su, sv, sw

    def step(self, u, v, w, un=None, vn=None, wn=None, dt=1.0, stream=None):
        """Fused forward Euler step: (un, vn, wn) = x + dt S(x), halos included."""
        un = self.empty() if un is None else un
        vn = self.empty() if vn is None else vn
        wn = self.empty() if wn is None else wn
        L.pw_advect_step(self.handle, self._check(u, "u"), self._check(v, "v"), self._check(w, "w"),
                         self._check(un, "un"), self._check(vn, "vn"), self._check(wn, "wn"), dt, _stream(stream))
        return un, vn, wn

    def advect_scalars(self, u, v, w, phis, sources=None, beta=0, stream=None):
        """PW sources of the cell-centred scalars phis (list of field tensors
        with halos filled) advected by (u, v, w); returns the list of sources."""
        phis = list(phis)
        sources = [self.empty_out() for _ in phis] if sources is None else list(sources)
        if len(sources) != len(phis):
            raise ValueError("one source tensor per scalar")
        L.pw_advect_scalars(self.handle, self._check(u, "u"), self._check(v, "v"), self._check(w, "w"),
                            [self._check(p, "phi") for p in phis],
                            [self._check(s, "sphi", True) for s in sources], beta, _stream(stream))
        return sources

    def advect_tvd(self, u, v, w, phis, dt, sources=None, beta=0, stream=None):
        """ULTIMATE-QUICKEST (flux-form, positivity-preserving) sources of the
        cell-centred scalars phis (halos filled) advected by (u, v, w) over a
        step dt; returns the list of sources."""
        phis = list(phis)
        sources = [self.empty_out() for _ in phis] if sources is None else list(sources)
        if len(sources) != len(phis):
            raise ValueError("one source tensor per scalar")
        L.pw_advect_tvd(self.handle, self._check(u, "u"), self._check(v, "v"), self._check(w, "w"),
                        [self._check(p, "phi") for p in phis],
                        [self._check(s, "sphi", True) for s in sources], dt, beta, _stream(stream))
        return sources

    def step_scalars(self, u, v, w, phis, outs=None, dt=1.0, stream=None):
        """Fused forward Euler step of the scalars: outs[a] = phis[a] + dt s(phis[a]),
        halos included; returns outs."""
        phis = list(phis)
        outs = [self.empty() for _ in phis] if outs is None else list(outs)
        if len(outs) != len(phis):
            raise ValueError("one output tensor per scalar")
        L.pw_advect_scalars_step(self.handle, self._check(u, "u"), self._check(v, "v"), self._check(w, "w"),
                                 [self._check(p, "phi") for p in phis], [self._check(o, "phin") for o in outs],
                                 dt, _stream(stream))
        return outs

    def adjoint(self, u, v, w, gsu, gsv, gsw, gu=None, gv=None, gw=None, alpha=1.0, beta=0, stream=None):
        gu = self.zeros() if gu is None else gu
        gv = self.zeros() if gv is None else gv
        gw = self.zeros() if gw is None else gw
        L.pw_advect_adjoint(self.handle, *(self._check(t, n) for t, n in ((u, "u"), (v, "v"), (w, "w"))),
                            *(self._check(t, n) for t, n in ((gsu, "gsu"), (gsv, "gsv"), (gsw, "gsw"))),
                            *(self._check(t, n) for t, n in ((gu, "gu"), (gv, "gv"), (gw, "gw"))),
                            alpha, beta, _stream(stream))
        return gu, gv, gw

    def euler_adjoint(self, u, v, w, gu_in, gv_in, gw_in, gu_out=None, gv_out=None, gw_out=None, dt=1.0,
                      stream=None):
        gu_out = self.zeros() if gu_out is None else gu_out
        gv_out = self.zeros() if gv_out is None else gv_out
        gw_out = self.zeros() if gw_out is None else gw_out
        L.pw_euler_adjoint(self.handle, *(self._check(t, "x") for t in (u, v, w)),
                           *(self._check(t, "g_in") for t in (gu_in, gv_in, gw_in)),
                           *(self._check(t, "g_out") for t in (gu_out, gv_out, gw_out)), dt, _stream(stream))
        return gu_out, gv_out, gw_out

    def euler(self, u, v, w, su, sv, sw, dt, stream=None):
        L.pw_euler(self.handle, self._check(u, "u"), self._check(v, "v"), self._check(w, "w"),
                   self._check(su, "su", True), self._check(sv, "sv", True), self._check(sw, "sw", True),
                   dt, _stream(stream))

    def residual_sums(self, u, v, w, su, sv, sw, stream=None):
        out = L.pw_residuals(self.handle, self._check(u, "u"), self._check(v, "v"), self._check(w, "w"),
                             self._check(su, "su", True), self._check(sv, "sv", True),
                             self._check(sw, "sw", True), _stream(stream))
        return np.array(out).reshape(3, 4)

    def residuals(self, u, v, w, su, sv, sw, stream=None):
        """((R_E u, v, w), (R_M u, v, w)) by pw_residual_ratios."""
        r = L.pw_residual_ratios(list(self.residual_sums(u, v, w, su, sv, sw, stream).reshape(-1)))
        return tuple(r[:3]), tuple(r[3:])

    def check_lid(self, w, stream=None):
        return L.pw_check_lid(self.handle, self._check(w, "w"), _stream(stream)) == L.PW_OK

    @property
    def algo(self):
        """The arithmetic this mesh uses: "split" or "native" (FP64), else "auto"."""
        return {L.PW_ALGO_AUTO: "auto", L.PW_ALGO_F64_NATIVE: "native",
                L.PW_ALGO_F64_SPLIT: "split"}[L.pw_mesh_algo(self.handle)]

    def device_status(self, clear=True, stream=None):
        return L.pw_mesh_device_status(self.handle, clear, _stream(stream))

    def set_tile(self, tile_j, tile_i):
        L.pw_mesh_set_tile(self.handle, tile_j, tile_i)

    def selftest_timeout(self, cycles=20_000_000, stream=None):
        L.pw_selftest_timeout(self.handle, cycles, _stream(stream))

    def get_tile(self):
        return L.pw_mesh_get_tile(self.handle)

    def autotune(self, u, v, w, su, sv, sw, cache_path=None, stream=None):
        return L.pw_autotune(self.handle, self._check(u, "u"), self._check(v, "v"), self._check(w, "w"),
                             self._check(su, "su", True), self._check(sv, "sv", True),
                             self._check(sw, "sw", True), cache_path, _stream(stream))


class Batch:
    """Many independent FP32 meshes advected in one persistent launch."""

    def __init__(self, meshes, stream=None):
        self.meshes = list(meshes)
        self.handle = L.pw_batch_create([m.handle for m in self.meshes], _stream(stream))
        self.fields = None

    def close(self):
        if getattr(self, "handle", None):
            L.pw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bind(self, fields, sources, stream=None):
        """fields: list of (u, v, w) per member; sources: list of (su, sv, sw)."""
        cols = [[], [], [], [], [], []]
        for m, f, s in zip(self.meshes, fields, sources):
            for q in range(3):
                cols[q].append(m._check(f[q], "uvw"[q]))
                cols[3 + q].append(m._check(s[q], "s" + "uvw"[q], True))
        L.pw_batch_set_fields(self.handle, *cols, _stream(stream))
        self.fields, self.sources = fields, sources

    def halo(self, stream=None):
        L.pw_batch_halo(self.handle, _stream(stream))

    def advect(self, beta=0, stream=None):
        L.pw_advect_batched(self.handle, beta, _stream(stream))

    def autotune(self, cache_path=None, stream=None):
        return L.pw_batch_autotune(self.handle, cache_path, _stream(stream))

    def set_tile(self, threads, tile_i, stream=None):
        L.pw_batch_set_tile(self.handle, threads, tile_i, _stream(stream))

    def set_schedule(self, persistent, stream=None):
        L.pw_batch_set_schedule(self.handle, persistent, _stream(stream))

    def status(self, clear=True, stream=None):
        return L.pw_batch_status(self.handle, clear, _stream(stream))


class Pipeline:
    """The halo fill + PW step on fields in host memory, with the copies
    overlapped slab by slab (pw_advect_host).  Host tensors are CPU tensors of
    the mesh shape and dtype, ideally pinned; the pipeline keeps device copies
    of the six fields."""

    def __init__(self, mesh, slab=0):
        self.mesh = mesh
        self.handle = L.pw_pipeline_create(mesh.handle, slab)
        self.slab, self.nslab = L.pw_pipeline_slab(self.handle)
        self._cb = None

    def close(self):
        if getattr(self, "handle", None):
            L.pw_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _host(self, t, name, out=False):
        m = self.mesh
        want = m.out_dtype if out else m.in_dtype
        if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
            raise TypeError(f"{name} must be a CPU tensor")
        if t.dtype != want:
            raise TypeError(f"{name} must be {want}, got {t.dtype}")
        if t.numel() != m.total or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with {m.total} elements (shape {m.shape})")
        return ctypes.c_void_p(t.data_ptr())

    def empty_host(self, out=False, pin=True):
        m = self.mesh
        return torch.zeros(m.shape, dtype=m.out_dtype if out else m.in_dtype, pin_memory=pin)

    def reserve_scalars(self, n):
        L.pw_pipeline_reserve_scalars(self.handle, n)

    def advect_host(self, u, v, w, su, sv, sw, beta=0, on_slab=None, stream=None, scalars=None, sources=None):
        """on_slab(i0, i1) runs on a CUDA host thread as each slab of the
        sources lands in the host arrays (it must not call CUDA).  scalars /
        sources: optional lists of host tensors (theta, q and their sources),
        advected by the same wind in the same step."""
        ins = [self._host(t, n) for t, n in ((u, "u"), (v, "v"), (w, "w"))]
        outs = [self._host(t, n, True) for t, n in ((su, "su"), (sv, "sv"), (sw, "sw"))]
        cb = None
        if on_slab is not None:
            cb = L.SLAB_FN(lambda user, i0, i1: on_slab(i0, i1))
        if scalars:
            if sources is None or len(sources) != len(scalars):
                raise ValueError("one host source tensor per scalar")
            ps = [self._host(t, "phi") for t in scalars]
            ss = [self._host(t, "sphi", True) for t in sources]
            L.pw_advect_host_scalars(self.handle, *ins, *outs, ps, ss, beta, cb, None, _stream(stream))
        else:
            L.pw_advect_host(self.handle, *ins, *outs, beta, cb, None, _stream(stream))
        self._cb = cb  # kept alive until the next call (which waits for these callbacks)

    def sync(self):
        L.pw_pipeline_sync(self.handle)

    def device_pointers(self):
        """Device addresses of the pipeline's copies of u, v, w, su, sv, sw
        (library layout, owned by the pipeline)."""
        return [p.value if hasattr(p, "value") else p for p in L.pw_pipeline_device_fields(self.handle)]
