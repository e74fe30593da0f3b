"""FP64 dense CPU oracle (ctypes wrapper around ``sbg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg use it to check and time the CUDA library; the
library itself never imports, links or calls anything here, and this package
shares no code with it.  The only inputs the two sides share come from the
``workloads`` package, which holds no arithmetic of the method.

Every function is the plain definition computed on the whole dense box; see
the C source for the passage of the paper each one follows.

SBG_ORACLE_LIB, when set, names a prebuilt library to load instead of
building ``sbg_oracle.c`` (the mutation tests point it at copies of the
oracle with one planted mistake each and check that a pin fails).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbg_oracle.c")
_LIB = os.environ.get("SBG_ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
FLT_EPSILON = float(np.finfo(np.float32).eps)

_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP, no FMA contraction)."""
    if os.environ.get("SBG_ORACLE_LIB"):
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        I = ctypes.c_int
        lib.oracle_num_threads.restype = I
        lib.oracle_active_mask.argtypes = [P, I64, ctypes.c_float, P]
        lib.oracle_fixed_mask.argtypes = [P, P, P, P]
        lib.oracle_surface_weight.argtypes = [P, P, I64, D, P]
        lib.oracle_stability_limit.argtypes = [P, P, I, P, P, D, D]
        lib.oracle_stability_limit.restype = D
        lib.oracle_step.argtypes = [P, P, P, P, I, P, P, P, D, P, P, D, P]
        lib.oracle_run.argtypes = [P, P, P, P, I, P, P, D, P, P, D, I64]
        lib.oracle_run.restype = I
        lib.oracle_rhs.argtypes = [P, P, P, P, I, P, P, P, P, D, P]
        lib.oracle_reduce.argtypes = [P, P, P, P, I, P, P, P, P, D, P]
        lib.oracle_effective_D.argtypes = [P, P, D, D, D, D, D, P, P, P]
        lib.oracle_steady_cg.argtypes = [P, P, P, P, D, P, D, I64, P]
        lib.oracle_steady_cg.restype = D
        lib.oracle_adjoint_step.argtypes = [P, P, P, P, I, P, P, P, P, D, P, P, D, P]
        lib.oracle_adjoint_run.argtypes = [P, P, P, P, I, P, P, D, P, P, D, I64, P, P, P, P]
        lib.oracle_adjoint_run.restype = I
        lib.oracle_eps_sigmoid.argtypes = [P, I64, D, D, D, D, P]
        lib.oracle_box_sum.argtypes = [P, P, P, P, P, P]
        lib.oracle_sussman.argtypes = [P, P, P, D, I64, P]
        lib.oracle_sussman.restype = I
        lib.oracle_upwind_grad.argtypes = [P, P, P, P]
        lib.oracle_step_inhom.argtypes = [P, P, P, P, P, P, P, D, D, D]
        lib.oracle_run_inhom.argtypes = [P, P, P, P, P, P, D, D, D, I64]
        lib.oracle_run_inhom.restype = I
        lib.oracle_reduce_inhom.argtypes = [P, P, P, P, P, P, D, D, P]
        lib.oracle_steady_cg_inhom.argtypes = [P, P, P, P, P, D, P, D, I64, P]
        lib.oracle_steady_cg_inhom.restype = D
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def eps_sigmoid(phi, d_min, d_max, g1, g2):
    """Eq. 6 per voxel: d_min + d_max / (1 + exp(-(g1 + g2 phi))), FP64."""
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    eps = np.empty(phi.shape, dtype=np.float64)
    _load().oracle_eps_sigmoid(_p(phi), int(phi.size), float(d_min), float(d_max), float(g1), float(g2),
                               _p(eps))
    return eps


@dataclass
class Problem:
    """A dense problem: phi plus the physics of one run.

    ``phys`` is any object with the fields of ``workloads.Physics``.
    Derived arrays (active, fixed, w) are computed here by the oracle.
    ``eps`` (optional, one species): a per-voxel diffusivity factor, the
    diffusivity being D * eps with face means (inhomogeneous diffusion, Eq. 6).
    """
    phi: np.ndarray
    phys: object
    eps: np.ndarray = None

    def __post_init__(self):
        lib = _load()
        self.phi = np.ascontiguousarray(self.phi, dtype=np.float32)
        nz, ny, nx = self.phi.shape
        self.dims = np.array([nx, ny, nz], dtype=np.int64)
        assert tuple(self.dims) == tuple(self.phys.dims), "phi shape does not match physics dims"
        self.n = int(nx * ny * nz)
        self.ns = int(self.phys.nspecies)
        self.dx = _f64(self.phys.dx)
        self.D = _f64(list(self.phys.D) + [0.0, 0.0])[:2].copy()
        self.decay = _f64(list(self.phys.decay) + [0.0, 0.0])[:2].copy()
        self.k = float(self.phys.k_surf)
        self.active = np.zeros(self.phi.shape, dtype=np.uint8)
        lib.oracle_active_mask(_p(self.phi), self.n, ctypes.c_float(FLT_EPSILON), _p(self.active))
        self.fixed = np.zeros(self.phi.shape, dtype=np.uint8)
        dirich = np.array([1 if f else 0 for f in self.phys.dirichlet], dtype=np.int32)
        lib.oracle_fixed_mask(_p(self.dims), _p(self.active), _p(dirich), _p(self.fixed))
        self.w = np.zeros(self.phi.shape, dtype=np.float64)
        lib.oracle_surface_weight(_p(self.phi), _p(self.active), self.n, float(self.phys.band_eps),
                                  _p(self.w))
        if self.eps is not None:
            assert self.ns == 1 and self.k == 0.0, "inhomogeneous diffusion: one species, no surface reaction"
            self.eps = _f64(self.eps).reshape(self.phi.shape).copy()

    # -- state helpers --------------------------------------------------------
    def shape_state(self, u):
        u = _f64(u).reshape((self.ns,) + self.phi.shape).copy()
        u *= self.active[None]  # inactive voxels carry 0
        return u

    # -- the method ---------------------------------------------------------
    def stability_limit(self) -> float:
        return float(_load().oracle_stability_limit(_p(self.dims), _p(self.dx), self.ns, _p(self.D),
                                                    _p(self.decay), self.k, float(self.phys.band_eps)))

    def step(self, u, dt=None, src=None):
        u = self.shape_state(u)
        out = np.empty_like(u)
        if self.eps is not None:
            assert src is None
            _load().oracle_step_inhom(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.eps), _p(u),
                                      _p(out), _p(self.dx), float(self.phys.dt if dt is None else dt),
                                      float(self.D[0]), float(self.decay[0]))
            return out
        src = None if src is None else _f64(src).reshape(u.shape)
        _load().oracle_step(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.w), self.ns,
                            _p(u), _p(out), _p(self.dx), float(self.phys.dt if dt is None else dt),
                            _p(self.D), _p(self.decay), self.k, _p(src))
        return out

    def run(self, u, nsteps, dt=None):
        u = self.shape_state(u)
        if self.eps is not None:
            rc = _load().oracle_run_inhom(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.eps), _p(u),
                                          _p(self.dx), float(self.phys.dt if dt is None else dt),
                                          float(self.D[0]), float(self.decay[0]), int(nsteps))
            if rc != 0:
                raise MemoryError("oracle_run_inhom: allocation failed")
            return u
        rc = _load().oracle_run(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.w), self.ns,
                                _p(u), _p(self.dx), float(self.phys.dt if dt is None else dt),
                                _p(self.D), _p(self.decay), self.k, int(nsteps))
        if rc != 0:
            raise MemoryError("oracle_run: allocation failed")
        return u

    def rhs(self, u):
        u = self.shape_state(u)
        out = np.empty_like(u)
        _load().oracle_rhs(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.w), self.ns,
                           _p(u), _p(self.dx), _p(self.D), _p(self.decay), self.k, _p(out))
        return out

    def reduce(self, u):
        """Per species: dict(mass, J_in, J_out, residual, n_active)."""
        u = self.shape_state(u)
        out = np.zeros(self.ns * 5)
        if self.eps is not None:
            _load().oracle_reduce_inhom(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.eps), _p(u),
                                        _p(self.dx), float(self.D[0]), float(self.decay[0]), _p(out))
            return [dict(zip(("mass", "J_in", "J_out", "residual", "n_active"), out[:5]))]
        _load().oracle_reduce(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.w), self.ns,
                              _p(u), _p(self.dx), _p(self.D), _p(self.decay), self.k, _p(out))
        keys = ("mass", "J_in", "J_out", "residual", "n_active")
        return [dict(zip(keys, out[s * 5:(s + 1) * 5])) for s in range(self.ns)]

    def effective_D(self, u):
        """(D_eff, tau, psi) from the x-face fluxes of species 0 (Eq. 2)."""
        r = self.reduce(u)[0]
        from workloads import FACE_XHI, FACE_XLO
        dC = abs(self.phys.face_value[FACE_XLO] - self.phys.face_value[FACE_XHI])
        d_eff, tau, psi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _load().oracle_effective_D(_p(self.dims), _p(self.dx), r["J_in"], r["J_out"], dC,
                                   float(self.D[0]), r["n_active"], ctypes.byref(d_eff),
                                   ctypes.byref(tau), ctypes.byref(psi))
        return d_eff.value, tau.value, psi.value

    def steady_cg(self, u0, tol=1e-13, maxit=100000):
        """FP64 CG steady state of species 0; returns (u, relres, iterations)."""
        u = self.shape_state(u0)[0].copy()
        iters = ctypes.c_int64()
        if self.eps is not None:
            rel = _load().oracle_steady_cg_inhom(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.eps),
                                                 _p(self.dx), float(self.D[0]), _p(u), float(tol), int(maxit),
                                                 ctypes.byref(iters))
            return u, float(rel), int(iters.value)
        rel = _load().oracle_steady_cg(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.dx),
                                       float(self.D[0]), _p(u), float(tol), int(maxit),
                                       ctypes.byref(iters))
        return u, float(rel), int(iters.value)

    def adjoint_step(self, u_n, lam_next, dt=None):
        u_n = self.shape_state(u_n)
        lam_next = _f64(lam_next).reshape(u_n.shape)
        lam = np.empty_like(u_n)
        grad = np.zeros(self.ns + 1)
        _load().oracle_adjoint_step(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.w),
                                    self.ns, _p(u_n), _p(lam_next), _p(lam), _p(self.dx),
                                    float(self.phys.dt if dt is None else dt), _p(self.D),
                                    _p(self.decay), self.k, _p(grad))
        return lam, grad

    def adjoint_run(self, u0, nsteps, lam_N, dt=None):
        """Returns (lambda^0, grad = [dL/dD_s..., dL/dk], u^N)."""
        u0 = self.shape_state(u0)
        lam_N = _f64(lam_N).reshape(u0.shape)
        lam0 = np.empty_like(u0)
        uN = np.empty_like(u0)
        grad = np.zeros(self.ns + 1)
        rc = _load().oracle_adjoint_run(_p(self.dims), _p(self.active), _p(self.fixed), _p(self.w),
                                        self.ns, _p(u0), _p(self.dx),
                                        float(self.phys.dt if dt is None else dt), _p(self.D),
                                        _p(self.decay), self.k, int(nsteps), _p(lam_N), _p(lam0),
                                        _p(grad), _p(uN))
        if rc != 0:
            raise MemoryError("oracle_adjoint_run: cannot store the state history")
        return lam0, grad, uN

    def box_sum(self, u, lo, hi, species=0):
        """(sum of u over the active voxels with lo <= (x, y, z) < hi, their count)."""
        u = self.shape_state(u)
        out = np.zeros(2)
        _load().oracle_box_sum(_p(self.dims), _p(self.active), _p(np.ascontiguousarray(u[species])),
                               _p(np.asarray(lo, dtype=np.int64)), _p(np.asarray(hi, dtype=np.int64)), _p(out))
        return float(out[0]), int(out[1])

    def frap_curve(self, u0, lo, hi, steps_per_sample, n_samples, species=0):
        """Simulated FRAP (Sec. 3.3): the box sum of ``u0`` and after every
        ``steps_per_sample`` steps, ``n_samples + 1`` values, and the box's
        active-voxel count."""
        u = self.shape_state(u0)
        sums = [self.box_sum(u, lo, hi, species)[0]]
        for _ in range(int(n_samples)):
            u = self.run(u, steps_per_sample)
            sums.append(self.box_sum(u, lo, hi, species)[0])
        return np.array(sums), self.box_sum(u, lo, hi, species)[1]

    # -- the gradient workload's loss -------------------------------------------
    def slab_mask(self, x_cut):
        m = np.zeros(self.phi.shape, dtype=bool)
        m[:, :, x_cut + 1:] = True
        return m & (self.active > 0)

    def slab_loss(self, u, x_cut):
        """Mean of species 0 over the active voxels with x > x_cut."""
        u = self.shape_state(u)
        m = self.slab_mask(x_cut)
        return float(u[0][m].sum() / m.sum())

    def slab_loss_seed(self, x_cut):
        """dL/du^N of slab_loss."""
        m = self.slab_mask(x_cut)
        lam = np.zeros((self.ns,) + self.phi.shape)
        lam[0][m] = 1.0 / m.sum()
        return lam


def frap_fit(t, f, t_ref, f_ref, s_lo=1e-3, s_hi=1.0):
    """Least-squares time-scale fit of a reference FRAP curve to a measured
    one (Sec. 3.3: the bulk-box curve fitted to the porous one): the s in
    [s_lo, s_hi] minimising sum_i (f_i - g(s t_i))^2, g the piecewise-linear
    interpolant of (t_ref, f_ref).  A dense scan, then scipy's bounded Brent
    search between the neighbours of the best scan point.  Returns (s, rss)."""
    from scipy.optimize import minimize_scalar

    t, f = _f64(t), _f64(f)
    t_ref, f_ref = _f64(t_ref), _f64(f_ref)

    def rss(s):
        return float(np.sum((f - np.interp(s * t, t_ref, f_ref)) ** 2))

    grid = np.linspace(s_lo, s_hi, 20001)
    vals = np.array([rss(s) for s in grid])
    k = int(np.argmin(vals))
    a, b = grid[max(k - 1, 0)], grid[min(k + 1, grid.size - 1)]
    r = minimize_scalar(rss, bounds=(a, b), method="bounded", options={"xatol": 1e-13 * s_hi})
    if r.fun <= vals[k]:
        return float(r.x), float(r.fun)
    return float(grid[k]), float(vals[k])


def sussman(phi0, dx=(1.0, 1.0, 1.0), cfl=0.3, iters=100):
    """Sussman redistancing (Sec. 2.1): ``iters`` forward-Euler iterations of
    the redistancing PDE with the smoothed sign and first-order Godunov
    differences; dalpha = cfl * min(dx).  phi0: dense [Nz, Ny, Nx]."""
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    nz, ny, nx = phi0.shape
    out = np.empty_like(phi0)
    rc = _load().oracle_sussman(_p(np.array([nx, ny, nz], dtype=np.int64)), _p(_f64(dx)), _p(phi0), float(cfl),
                                int(iters), _p(out))
    if rc != 0:
        raise MemoryError("oracle_sussman: allocation failed")
    return out


def upwind_grad(phi, dx=(1.0, 1.0, 1.0)):
    """The Godunov |grad phi| per voxel for the sign of phi there."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    nz, ny, nx = phi.shape
    out = np.empty_like(phi)
    _load().oracle_upwind_grad(_p(np.array([nx, ny, nz], dtype=np.int64)), _p(_f64(dx)), _p(phi), _p(out))
    return out
