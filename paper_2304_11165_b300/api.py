"""Python binding over the C ABI (argument marshalling only: every step of the
path runs in the library's CUDA kernels).  Device buffers, streams and
autograd come from PyTorch; dense inputs may be numpy arrays (host) or torch
tensors (host or CUDA)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import NRED, Params, check, load

_DTYPES = {"f32": _abi.SBG_F32, "f64": _abi.SBG_F64, "f32x2": _abi.SBG_F32X2, "f32r": _abi.SBG_F32R}
_ORDERS = {"tiled": _abi.SBG_ORDER_TILED, "planes": _abi.SBG_ORDER_PLANES}


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dense_ptr(a, allow_f32=True):
    """(pointer, dtype code, on_device, keepalive) for a dense array or tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                a = a.contiguous()
            if a.dtype == torch.float64:
                code = _abi.SBG_F64
            elif a.dtype == torch.float32 and allow_f32:
                code = _abi.SBG_F32
            else:
                raise TypeError("dense tensors must be float32 or float64")
            return ctypes.c_void_p(a.data_ptr()), code, int(a.is_cuda), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a)
    if arr.dtype == np.float64:
        code = _abi.SBG_F64
    elif arr.dtype == np.float32 and allow_f32:
        code = _abi.SBG_F32
    else:
        arr = arr.astype(np.float64)
        code = _abi.SBG_F64
    return arr.ctypes.data_as(ctypes.c_void_p), code, 0, arr


def make_params(phys, allow_unstable: bool = False, dt=None) -> Params:
    """Params from any object with the fields of ``workloads.Physics``."""
    p = Params()
    for a in range(3):
        p.dx[a] = float(phys.dx[a])
    p.dt = float(phys.dt if dt is None else dt)
    p.nspecies = int(phys.nspecies)
    for f in range(6):
        p.face_type[f] = _abi.SBG_FACE_DIRICHLET if phys.dirichlet[f] else _abi.SBG_FACE_NOFLUX
        p.face_value[f] = float(phys.face_value[f])
    D = list(phys.D) + [0.0, 0.0]
    decay = list(phys.decay) + [0.0, 0.0]
    for s in range(2):
        p.D[s] = float(D[s])
        p.decay[s] = float(decay[s])
    p.k_surf = float(phys.k_surf)
    p.allow_unstable = int(bool(allow_unstable))
    return p


def stability_limit(params: Params, dims, band_eps: float = 1.0) -> float:
    d = (ctypes.c_int64 * 3)(*[int(x) for x in dims])
    return float(load().sbg_stability_limit(ctypes.byref(params), d, float(band_eps)))


class Grid:
    """A sparse block grid built on the device from one or more phi fields."""

    def __init__(self, phi=None, block: int = 8, eps_mask: float = 0.0, band_eps: float = 1.0,
                 stream=None, order: str = "tiled", _handle=None, _keep=None):
        lib = load()
        self._lib = lib
        if _handle is not None:
            self.handle = _handle
        else:
            opts = _abi.BuildOpts(block, 0, eps_mask, band_eps, _ORDERS[order])
            ptr, code, on_dev, keep = _phi_ptr(phi)
            opts.phi_on_device = on_dev
            nz, ny, nx = phi.shape
            dims = (ctypes.c_int64 * 3)(nx, ny, nz)
            h = ctypes.c_void_p()
            check(lib.sbg_build(ptr, dims, ctypes.byref(opts), _stream_handle(stream), ctypes.byref(h)))
            self.handle = h
        self._refresh_info()

    @classmethod
    def batch(cls, phis, block: int = 8, eps_mask: float = 0.0, band_eps: float = 1.0, stream=None,
              order: str = "tiled"):
        lib = load()
        n = len(phis)
        ptrs = (ctypes.c_void_p * n)()
        dims = (ctypes.c_int64 * (3 * n))()
        keep = []
        on_dev = None
        for i, phi in enumerate(phis):
            ptr, code, dev, k = _phi_ptr(phi)
            if on_dev is None:
                on_dev = dev
            elif on_dev != dev:
                raise ValueError("all phi fields must live on the same side (host or device)")
            keep.append(k)
            ptrs[i] = ptr
            nz, ny, nx = phi.shape
            dims[3 * i:3 * i + 3] = [nx, ny, nz]
        opts = _abi.BuildOpts(block, on_dev or 0, eps_mask, band_eps, _ORDERS[order])
        h = ctypes.c_void_p()
        check(lib.sbg_build_batch(n, ptrs, dims, ctypes.byref(opts), _stream_handle(stream),
                                  ctypes.byref(h)))
        return cls(_handle=h)

    def _refresh_info(self):
        info = _abi.GridInfo()
        check(self._lib.sbg_grid_info(self.handle, ctypes.byref(info)))
        self.info = {f: (list(getattr(info, f)) if f == "dims" else getattr(info, f))
                     for f, _ in _abi.GridInfo._fields_}
        self.block = info.block
        self.n_geoms = info.n_geoms
        self.n_blocks = info.n_blocks
        self.n_active = info.n_active

    def geometry_info(self):
        n = self.n_geoms
        na, bb, bc = (np.zeros(n, np.int64) for _ in range(3))
        check(self._lib.sbg_grid_geometry_info(self.handle, na.ctypes.data_as(ctypes.c_void_p),
                                               bb.ctypes.data_as(ctypes.c_void_p),
                                               bc.ctypes.data_as(ctypes.c_void_p)))
        return na, bb, bc

    def set_diffusivity(self, eps, geom: int = 0, stream=None):
        """Per-voxel diffusivity factor (inhomogeneous diffusion of one species:
        D_0 * eps with face means); eps: dense [Nz, Ny, Nx], numpy or torch."""
        ptr, code, on_dev, keep = _dense_ptr(eps)
        check(self._lib.sbg_grid_set_diffusivity(self.handle, geom, ptr, code, on_dev, _stream_handle(stream)))
        return self

    def set_diffusivity_sigmoid(self, phi, d_min, d_max, gamma1, gamma2, geom: int = 0, stream=None):
        """The factor from phi by Eq. 6: d_min + d_max / (1 + exp(-(gamma1 + gamma2 phi)))."""
        if isinstance(phi, np.ndarray):
            arr = np.ascontiguousarray(phi, dtype=np.float32)
            ptr, on_dev, keep = arr.ctypes.data_as(ctypes.c_void_p), 0, arr
        else:
            keep = phi.contiguous().float()
            ptr, on_dev = ctypes.c_void_p(keep.data_ptr()), int(keep.is_cuda)
        check(self._lib.sbg_grid_set_diffusivity_sigmoid(self.handle, geom, ptr, on_dev, float(d_min), float(d_max),
                                                         float(gamma1), float(gamma2), _stream_handle(stream)))
        return self

    def clear_diffusivity(self):
        check(self._lib.sbg_grid_clear_diffusivity(self.handle))
        return self

    def tables(self):
        nbr = np.zeros((self.n_blocks, 26), np.int32)
        blocks = np.zeros((self.n_blocks, 4), np.int32)
        check(self._lib.sbg_grid_tables(self.handle, nbr.ctypes.data_as(ctypes.c_void_p),
                                        blocks.ctypes.data_as(ctypes.c_void_p)))
        return nbr, blocks

    def close(self):
        if getattr(self, "handle", None):
            self._lib.sbg_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _phi_ptr(phi):
    try:
        import torch
        if isinstance(phi, torch.Tensor):
            t = phi.contiguous().to(torch.float32)
            return ctypes.c_void_p(t.data_ptr()), _abi.SBG_F32, int(t.is_cuda), t
    except ImportError:
        pass
    arr = np.ascontiguousarray(phi, dtype=np.float32)
    return arr.ctypes.data_as(ctypes.c_void_p), _abi.SBG_F32, 0, arr


class State:
    """Species fields of one grid, in block layout, with their ping-pong partner."""

    def __init__(self, grid: Grid, nspecies: int = 1, dtype: str = "f32"):
        self.grid = grid
        self.nspecies = nspecies
        self.dtype = dtype
        self._lib = grid._lib
        h = ctypes.c_void_p()
        check(self._lib.sbg_state_create(grid.handle, nspecies, _DTYPES[dtype], ctypes.byref(h)))
        self.handle = h

    def set(self, dense, species: int = 0, geom: int = 0, stream=None):
        ptr, code, on_dev, keep = _dense_ptr(dense)
        check(self._lib.sbg_state_set(self.grid.handle, self.handle, geom, species, ptr, code, on_dev,
                                      _stream_handle(stream)))
        return self

    def set_all(self, dense, geom: int = 0, stream=None):
        """dense: [S, Nz, Ny, Nx] (or [Nz, Ny, Nx] for one species)."""
        if self.nspecies == 1 and dense.ndim == 3:
            return self.set(dense, 0, geom, stream)
        for s in range(self.nspecies):
            self.set(dense[s], s, geom, stream)
        return self

    def get(self, species: int = 0, geom: int = 0, out=None, stream=None):
        """Dense [Nz, Ny, Nx] copy (float64 numpy by default; or into `out`)."""
        dims = self.grid.info["dims"] if geom == 0 else None
        if out is None:
            if dims is None:
                raise ValueError("pass `out` for geometries other than 0")
            out = np.zeros((dims[2], dims[1], dims[0]), np.float64)
        ptr, code, on_dev, keep = _dense_ptr(out)
        check(self._lib.sbg_state_get(self.grid.handle, self.handle, geom, species, ptr, code, on_dev,
                                      _stream_handle(stream)))
        return out

    def get_all(self, geom: int = 0):
        return np.stack([self.get(s, geom) for s in range(self.nspecies)])

    def set_kernel(self, variant: str = "auto", ctas_per_sm: int = 0):
        code = {"auto": _abi.SBG_KERNEL_AUTO, "plain": _abi.SBG_KERNEL_PLAIN,
                "pipelined": _abi.SBG_KERNEL_PIPELINED,
                "prefetch": _abi.SBG_KERNEL_PIPELINED_PREFETCH, "async": _abi.SBG_KERNEL_PIPELINED_ASYNC,
                "stream": _abi.SBG_KERNEL_STREAM, "wave": _abi.SBG_KERNEL_WAVE,
                "wave4": _abi.SBG_KERNEL_WAVE4}[variant]
        check(self._lib.sbg_state_set_kernel(self.handle, code, int(ctas_per_sm)))
        return self

    def copy_from(self, other: "State", stream=None):
        check(self._lib.sbg_state_copy(self.handle, other.handle, _stream_handle(stream)))
        return self

    def step(self, params: Params, nsteps: int, stream=None):
        check(self._lib.sbg_step(self.grid.handle, self.handle, ctypes.byref(params), int(nsteps),
                                 _stream_handle(stream)))
        return self

    def set_source(self, dense, species: int = 0, geom: int = 0, stream=None):
        """Spatial part S_s(x) of an external source a_n S_s(x) (dense [Nz, Ny, Nx])."""
        ptr, code, on_dev, keep = _dense_ptr(dense)
        check(self._lib.sbg_state_set_source(self.grid.handle, self.handle, geom, species, ptr, code, on_dev,
                                             _stream_handle(stream)))
        return self

    def clear_source(self):
        check(self._lib.sbg_state_clear_source(self.handle))
        return self

    def step_source(self, params: Params, factors, stream=None):
        """len(factors) steps; step n adds dt * factors[n] * S_s(x)."""
        f = np.ascontiguousarray(factors, dtype=np.float64)
        check(self._lib.sbg_step_source(self.grid.handle, self.handle, ctypes.byref(params), int(f.size),
                                        f.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)))
        return self

    _RED_KEYS = ("mass", "J_in", "J_out", "residual", "min", "max", "nonfinite", "n_active")

    def reduce(self, params: Params, geom: int = 0, stream=None):
        out = np.zeros(self.nspecies * NRED)
        check(self._lib.sbg_reduce(self.grid.handle, self.handle, ctypes.byref(params), geom,
                                   out.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)))
        return self.parse_reduction(out)

    def parse_reduction(self, out):
        """Per-species dicts from an array of nspecies * SBG_NRED results."""
        out = np.asarray(out, dtype=np.float64)
        return [dict(zip(self._RED_KEYS, out[s * NRED:(s + 1) * NRED])) for s in range(self.nspecies)]

    def reduce_async(self, params: Params, out, geom: int = 0, stream=None):
        """Enqueue the reductions (``sbg_reduce_async``) into ``out``: a float64
        torch tensor of nspecies * SBG_NRED elements, page-locked host memory
        or device memory; read it (``parse_reduction``) once the stream has
        passed this call."""
        check(self._lib.sbg_reduce_async(self.grid.handle, self.handle, ctypes.byref(params), geom,
                                         ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def check_async(self, params: Params, out, geom: int = 0, stream=None):
        """Enqueue the monitoring check (``sbg_check_async``: every scalar of
        ``reduce_async`` but the residual, which reads NaN) into ``out``, with
        the same rules as ``reduce_async``."""
        check(self._lib.sbg_check_async(self.grid.handle, self.handle, ctypes.byref(params), geom,
                                        ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def box_sum(self, lo, hi, species: int = 0, geom: int = 0, stream=None):
        """(sum of u over the active voxels with lo <= (x, y, z) < hi, their count)."""
        lo_a = np.asarray(lo, dtype=np.int64)
        hi_a = np.asarray(hi, dtype=np.int64)
        out = np.zeros(2)
        check(self._lib.sbg_reduce_box(self.grid.handle, self.handle, geom, species,
                                       lo_a.ctypes.data_as(ctypes.c_void_p), hi_a.ctypes.data_as(ctypes.c_void_p),
                                       out.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)))
        return float(out[0]), int(out[1])

    def frap_curve(self, params: Params, lo, hi, steps_per_sample: int, n_samples: int, species: int = 0,
                   geom: int = 0, stream=None):
        """Box sums before the first step and after every ``steps_per_sample``
        steps (``n_samples + 1`` values) and the box's active-voxel count."""
        lo_a = np.asarray(lo, dtype=np.int64)
        hi_a = np.asarray(hi, dtype=np.int64)
        sums = np.zeros(int(n_samples) + 1)
        count = ctypes.c_int64(0)
        check(self._lib.sbg_frap_curve(self.grid.handle, self.handle, ctypes.byref(params), geom, species,
                                       lo_a.ctypes.data_as(ctypes.c_void_p), hi_a.ctypes.data_as(ctypes.c_void_p),
                                       int(steps_per_sample), int(n_samples), sums.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.byref(count), _stream_handle(stream)))
        return sums, int(count.value)

    def frap_recovery(self, params: Params, lo, hi, steps_per_sample: int, n_samples: int, species: int = 0,
                      geom: int = 0, stream=None):
        """(t, F, n_box): the recovery curve of the box normalised by its own
        equilibrium (``sbg_frap_recovery``)."""
        lo_a = np.asarray(lo, dtype=np.int64)
        hi_a = np.asarray(hi, dtype=np.int64)
        t = np.zeros(int(n_samples) + 1)
        F = np.zeros(int(n_samples) + 1)
        count = ctypes.c_int64(0)
        v = ctypes.c_void_p
        check(self._lib.sbg_frap_recovery(self.grid.handle, self.handle, ctypes.byref(params), geom, species,
                                          lo_a.ctypes.data_as(v), hi_a.ctypes.data_as(v), int(steps_per_sample),
                                          int(n_samples), t.ctypes.data_as(v), F.ctypes.data_as(v),
                                          ctypes.byref(count), _stream_handle(stream)))
        return t, F, int(count.value)

    def effective_D(self, params: Params, geom: int = 0, stream=None):
        d, t, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(self._lib.sbg_effective_D(self.grid.handle, self.handle, ctypes.byref(params), geom,
                                        ctypes.byref(d), ctypes.byref(t), ctypes.byref(p),
                                        _stream_handle(stream)))
        return d.value, t.value, p.value

    def run_to_steady(self, params: Params, tol: float, check_every: int = 1000,
                      max_steps: int = 10 ** 9, stream=None, raise_on_max=True):
        steps, rel = ctypes.c_int64(), ctypes.c_double()
        rc = self._lib.sbg_run_to_steady(self.grid.handle, self.handle, ctypes.byref(params), float(tol),
                                         int(check_every), int(max_steps), ctypes.byref(steps),
                                         ctypes.byref(rel), _stream_handle(stream))
        if rc != _abi.SBG_OK and not (rc == _abi.SBG_ERR_NOT_CONVERGED and not raise_on_max):
            check(rc)
        return steps.value, rel.value

    def batch_run_to_steady(self, params: Params, tol: float, check_every: int = 128,
                            max_steps: int = 10 ** 9, stream=None, raise_on_max=True):
        """All geometries of a batched grid to steady state; returns (steps[g], rel[g])."""
        n = self.grid.n_geoms
        steps = np.zeros(n, np.int64)
        rel = np.zeros(n)
        rc = self._lib.sbg_batch_run_to_steady(self.grid.handle, self.handle, ctypes.byref(params), float(tol),
                                               int(check_every), int(max_steps),
                                               steps.ctypes.data_as(ctypes.c_void_p),
                                               rel.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream))
        if rc != _abi.SBG_OK and not (rc == _abi.SBG_ERR_NOT_CONVERGED and not raise_on_max):
            check(rc)
        return steps, rel

    def close(self):
        if getattr(self, "handle", None):
            self._lib.sbg_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def frap_fit(t, f, t_ref, f_ref, s_lo: float = 1e-3, s_hi: float = 1.0):
    """(scale s, residual sum of squares) of the least-squares fit of the
    reference curve g = interp(t_ref, f_ref) to (t, f) over g(s t)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    t_ref = np.ascontiguousarray(t_ref, dtype=np.float64)
    f_ref = np.ascontiguousarray(f_ref, dtype=np.float64)
    if t.shape != f.shape or t_ref.shape != f_ref.shape:
        raise ValueError("frap_fit: times and values differ in length")
    scale = ctypes.c_double(0.0)
    rss = ctypes.c_double(0.0)
    v = ctypes.c_void_p
    check(load().sbg_frap_fit(t.ctypes.data_as(v), f.ctypes.data_as(v), t.size, t_ref.ctypes.data_as(v),
                              f_ref.ctypes.data_as(v), t_ref.size, float(s_lo), float(s_hi), ctypes.byref(scale),
                              ctypes.byref(rss)))
    return scale.value, rss.value


def frap_effective_D(t, F, t_ref, F_ref, D_ref: float, s_lo: float = 1e-3, s_hi: float = 1.0):
    """(D_eff, tau, scale, rss) of the FRAP fit (``sbg_frap_effective_D``)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (t, F, t_ref, F_ref)]
    if arrs[0].shape != arrs[1].shape or arrs[2].shape != arrs[3].shape:
        raise ValueError("frap_effective_D: times and values differ in length")
    d, tau, sc, rss = (ctypes.c_double(0.0) for _ in range(4))
    v = ctypes.c_void_p
    check(load().sbg_frap_effective_D(arrs[0].ctypes.data_as(v), arrs[1].ctypes.data_as(v), arrs[0].size,
                                      arrs[2].ctypes.data_as(v), arrs[3].ctypes.data_as(v), arrs[2].size,
                                      float(D_ref), float(s_lo), float(s_hi), ctypes.byref(d), ctypes.byref(tau),
                                      ctypes.byref(sc), ctypes.byref(rss)))
    return d.value, tau.value, sc.value, rss.value


def redistance(phi0, dx=(1.0, 1.0, 1.0), cfl: float = 0.3, max_iter: int = 200, tol: float = 0.0,
               band: float = 2.0, check_every: int = 16, stream=None):
    """Sussman redistancing of a dense [Nz, Ny, Nx] level set on the device
    (``sbg_redistance``).  A float32/float64 numpy array gives a numpy array
    back, a CUDA tensor a CUDA tensor of the same dtype.  Returns
    (phi, iterations, last tested residual)."""
    try:
        import torch
        is_tensor = isinstance(phi0, torch.Tensor)
    except ImportError:
        is_tensor = False
    if is_tensor:
        src = phi0.contiguous()
        if src.dtype not in (torch.float32, torch.float64) or not src.is_cuda:
            raise TypeError("redistance: CUDA float32/float64 tensors only")
        out = torch.empty_like(src)
        code = _abi.SBG_F64 if src.dtype == torch.float64 else _abi.SBG_F32
        pin, pout, on_dev = ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1
    else:
        src = np.ascontiguousarray(phi0)
        if src.dtype not in (np.float32, np.float64):
            src = src.astype(np.float64)
        out = np.empty_like(src)
        code = _abi.SBG_F64 if src.dtype == np.float64 else _abi.SBG_F32
        pin, pout, on_dev = src.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p), 0
    nz, ny, nx = src.shape
    dims = (ctypes.c_int64 * 3)(nx, ny, nz)
    dxa = (ctypes.c_double * 3)(*[float(d) for d in dx])
    opts = _abi.RedistOpts(float(cfl), int(max_iter), float(tol), float(band), int(check_every))
    iters = ctypes.c_int64(0)
    res = ctypes.c_double(0.0)
    check(load().sbg_redistance(dims, dxa, pin, pout, code, on_dev, ctypes.byref(opts), ctypes.byref(iters),
                                ctypes.byref(res), _stream_handle(stream)))
    return out, iters.value, res.value
