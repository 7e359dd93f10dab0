"""ctypes binding of the C interface in include/mf.h (argument marshalling only).

Every computation runs in the CUDA library libmf.so; this module converts Python and torch
arguments to plain pointers and sizes.  PyTorch provides the device memory (the workspace and
state tensors) and the current CUDA stream.  Importing the module does not load the library;
the first call does, and fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmf.so")

MF_OK, MF_ERR_ARG, MF_ERR_CUDA, MF_ERR_NOCONV, MF_ERR_NONFINITE = 0, 1, 2, 3, 4
MF_ERR_STEP_UNDERFLOW, MF_ERR_WORKSPACE, MF_ERR_BARRIER = 5, 6, 7
MF_READ_HZ, MF_READ_MOMENT, MF_READ_J, MF_READ_E = 0, 1, 2, 3
STATUS_NAMES = {0: "MF_OK", 1: "MF_ERR_ARG", 2: "MF_ERR_CUDA", 3: "MF_ERR_NOCONV",
                4: "MF_ERR_NONFINITE", 5: "MF_ERR_STEP_UNDERFLOW", 6: "MF_ERR_WORKSPACE",
                7: "MF_ERR_BARRIER"}

# every entry point declared in include/mf.h
EXPORTS = ["mf_default_params", "mf_workspace_bytes", "mf_create", "mf_rhs", "mf_rhs_ex",
           "mf_reset_warm", "mf_set_state", "mf_get_state", "mf_advance", "mf_step",
           "mf_run_ramp", "mf_readout", "mf_readout_of", "mf_get_info", "mf_get_log",
           "mf_last_error", "mf_destroy", "mf_film_rhs_noalloc", "mf_advance_batch",
           "mf_autotune", "mf_batch_plan", "mf_checkpoint_bytes", "mf_checkpoint_save",
           "mf_checkpoint_restore", "mf_film_outside_vjp", "mf_film_rhs_vjp",
           "mf_film_solve_gradient_work_bytes", "mf_film_solve_gradient", "mf_set_jc_map",
           "mf_set_knot_values", "mf_set_barrier_timeout", "mf_film_rhs_vjp_warm"]


class mf_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("mask", ctypes.POINTER(ctypes.c_uint8)), ("jc_map", ctypes.POINTER(ctypes.c_double)),
        ("jc", ctypes.c_double), ("n", ctypes.c_double), ("e0", ctypes.c_double),
        ("rho_out", ctypes.c_double), ("sigma", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("iter_tol", ctypes.c_double), ("iter_max", ctypes.c_int), ("precision", ctypes.c_int),
        ("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("h0", ctypes.c_double),
        ("h_min", ctypes.c_double),
        ("he_t", ctypes.POINTER(ctypes.c_double)), ("he_v", ctypes.POINTER(ctypes.c_double)),
        ("he_knots", ctypes.c_int), ("he_sin_amp", ctypes.c_double),
        ("he_sin_period", ctypes.c_double), ("he_dir", ctypes.c_double * 3),
        ("gamma", ctypes.c_double), ("b0", ctypes.c_double),
    ]


class mf_step_log(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("h", ctypes.c_double), ("t_new", ctypes.c_double),
                ("err", ctypes.c_double), ("outcome", ctypes.c_int),
                ("iters", ctypes.c_int * 4), ("pad", ctypes.c_int)]


class mf_info(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("h", ctypes.c_double),
                ("n_attempts", ctypes.c_longlong), ("n_accepted", ctypes.c_longlong),
                ("n_rejected", ctypes.c_longlong), ("n_rhs", ctypes.c_longlong),
                ("n_iters", ctypes.c_longlong), ("n_noconv", ctypes.c_longlong),
                ("log_count", ctypes.c_longlong), ("last_iters", ctypes.c_int),
                ("last_r", ctypes.c_double), ("last_err", ctypes.c_double),
                ("grid", ctypes.c_int), ("threads", ctypes.c_int), ("smem_bytes", ctypes.c_int),
                ("rows_per_item", ctypes.c_int), ("workspace_used", ctypes.c_longlong)]


class mf_tuning(ctypes.Structure):
    _fields_ = [("rows_per_item", ctypes.c_int), ("zs_per_item", ctypes.c_int),
                ("grid", ctypes.c_int), ("candidates", ctypes.c_int),
                ("ms_per_rhs", ctypes.c_double), ("ms_per_rhs_default", ctypes.c_double)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libmf.so (built by paper_1801_04869_gb300/build.py); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_1801_04869_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, dp, ip = ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_int)
    sig = {
        "mf_default_params": (None, [P(mf_params)]),
        "mf_workspace_bytes": (ctypes.c_size_t, [P(mf_params)]),
        "mf_create": (ctypes.c_int, [P(mf_params), vp, ctypes.c_size_t, vp, P(vp)]),
        "mf_rhs": (ctypes.c_int, [vp, ctypes.c_double, vp, vp, ip]),
        "mf_rhs_ex": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int, vp, vp, ctypes.c_int, ip]),
        "mf_reset_warm": (ctypes.c_int, [vp]),
        "mf_set_barrier_timeout": (ctypes.c_int, [vp, ctypes.c_double]),
        "mf_set_state": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, vp]),
        "mf_get_state": (ctypes.c_int, [vp, dp, dp, vp]),
        "mf_advance": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_longlong]),
        "mf_advance_batch": (ctypes.c_int, [P(vp), ctypes.c_int, dp, ctypes.c_longlong, ip]),
        "mf_step": (ctypes.c_int, [vp, ctypes.c_double, ip]),
        "mf_run_ramp": (ctypes.c_int, [vp, ctypes.c_int, dp, dp, vp]),
        "mf_readout": (ctypes.c_int, [vp, ctypes.c_int, vp]),
        "mf_readout_of": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, vp, vp]),
        "mf_get_info": (ctypes.c_int, [vp, P(mf_info)]),
        "mf_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, P(mf_tuning)]),
        "mf_batch_plan": (ctypes.c_int, [ctypes.c_int, ip, ip, ip, dp, ctypes.c_int, ip, ip, ip]),
        "mf_checkpoint_bytes": (ctypes.c_size_t, [vp]),
        "mf_checkpoint_save": (ctypes.c_int, [vp, vp]),
        "mf_checkpoint_restore": (ctypes.c_int, [vp, vp]),
        "mf_film_outside_vjp": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, dp]),
        "mf_film_rhs_vjp": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp, vp, dp]),
        "mf_film_rhs_vjp_warm": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, dp]),
        "mf_film_solve_gradient_work_bytes": (ctypes.c_size_t, [vp, ctypes.c_int, ctypes.c_int]),
        "mf_set_jc_map": (ctypes.c_int, [vp, vp]),
        "mf_set_knot_values": (ctypes.c_int, [vp, dp, ctypes.c_int]),
        "mf_film_solve_gradient": (ctypes.c_int, [vp, ctypes.c_int, dp, dp, ip, ctypes.c_int, vp, vp,
                                                  vp, vp, ctypes.c_size_t, vp, dp, ctypes.c_int, vp,
                                                  vp, dp]),
        "mf_get_log": (ctypes.c_int, [vp, P(mf_step_log), ctypes.c_longlong, P(ctypes.c_longlong)]),
        "mf_last_error": (ctypes.c_char_p, [vp]),
        "mf_destroy": (None, [vp]),
        "mf_film_rhs_noalloc": (ctypes.c_int, [P(mf_params), ctypes.c_double, vp, vp, ctypes.c_int,
                                               vp, ip, ctypes.c_char_p, ctypes.c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class MFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _dptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _arr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Problem:
    """A problem set up in a torch-allocated device workspace (see mf_create in mf.h)."""

    def __init__(self, *, dim: int, nx: int, ny: int, nz: int = 1, Lx: float, Ly: float,
                 Lz: float = 0.0, mask, n: float, rho_out: float, precision: int = 0,
                 jc: float = 1.0, jc_map=None, e0: float = 1.0, sigma: float = 0.0,
                 lam: float = 0.7, iter_tol: float = 2e-4, iter_max: int = 1000,
                 rtol: float = 1e-6, atol: float = 1e-6, h0: float = 0.0, h_min: float = 1e-12,
                 he_knots=None, he_sin=None, he_dir=(0.0, 0.0, 1.0), gamma: float = 1.0,
                 b0: float = 0.0, device=None, stream=None):
        import torch
        lib = load()
        self.lib = lib
        p = mf_params()
        lib.mf_default_params(ctypes.byref(p))
        self._keep = []
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self._keep.append(m)
        p.dim, p.nx, p.ny, p.nz = dim, nx, ny, (1 if dim == 2 else nz)
        p.Lx, p.Ly, p.Lz = Lx, Ly, Lz
        p.mask = _arr(m, ctypes.c_uint8)
        if jc_map is not None:
            jm = np.ascontiguousarray(jc_map, dtype=np.float64).reshape(-1)
            self._keep.append(jm)
            p.jc_map = _arr(jm, ctypes.c_double)
        p.jc, p.n, p.e0, p.rho_out, p.sigma = jc, n, e0, rho_out, sigma
        p.lambda_, p.iter_tol, p.iter_max, p.precision = lam, iter_tol, iter_max, precision
        p.rtol, p.atol, p.h0, p.h_min = rtol, atol, h0, h_min
        if he_knots is not None:
            kt = np.ascontiguousarray(he_knots[0], dtype=np.float64)
            kv = np.ascontiguousarray(he_knots[1], dtype=np.float64)
            self._keep += [kt, kv]
            p.he_t, p.he_v, p.he_knots = _arr(kt, ctypes.c_double), _arr(kv, ctypes.c_double), len(kt)
        else:
            amp, per = he_sin if he_sin is not None else (0.0, 1.0)
            p.he_knots, p.he_sin_amp, p.he_sin_period = 0, amp, per
        p.he_dir[0], p.he_dir[1], p.he_dir[2] = he_dir
        p.gamma, p.b0 = gamma, b0
        self.params = p
        nbytes = lib.mf_workspace_bytes(ctypes.byref(p))
        if nbytes == 0:
            raise MFError(MF_ERR_ARG, "invalid parameters (mf_workspace_bytes returned 0)")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        off = (-base) % 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        st = lib.mf_create(ctypes.byref(p), ctypes.c_void_p(base + off), ctypes.c_size_t(nbytes),
                           ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != MF_OK:
            raise MFError(st, "mf_create failed")
        self.h = h
        self.dim, self.nx, self.ny, self.nz = dim, nx, ny, p.nz
        self.state_len = nx * ny * (1 if dim == 2 else 3 * p.nz)

    # -- helpers -----------------------------------------------------------------------------
    def _f64(self, t, n: int, name: str) -> ctypes.c_void_p:
        """Device pointer of `t`, a contiguous float64 tensor of at least n values on the
        problem's device (None: NULL).  The library takes bare pointers and cannot check a
        buffer's length, so a short or misplaced tensor is refused here."""
        if t is None:
            return ctypes.c_void_p(0)
        import torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64:
            raise TypeError(f"{name}: a float64 torch tensor is needed, got "
                            f"{getattr(t, 'dtype', type(t).__name__)}")
        if not t.is_cuda or t.device.index != self.device.index:
            raise ValueError(f"{name}: the tensor must be on {self.device}, it is on {t.device}")
        if not t.is_contiguous():
            raise ValueError(f"{name}: the tensor must be contiguous")
        if t.numel() < n:
            raise ValueError(f"{name}: {n} values are needed, the tensor has {t.numel()}")
        return ctypes.c_void_p(t.data_ptr())

    def _readout_len(self, what: int) -> int:
        ncell = self.nx * self.ny * self.nz
        if what == MF_READ_HZ:
            return ncell
        return (2 if self.dim == 2 and what == MF_READ_E else 3) * ncell

    def _blob(self, t, name: str) -> ctypes.c_void_p:
        n = self.lib.mf_checkpoint_bytes(self.h)
        if t.numel() * t.element_size() < n or not t.is_contiguous():
            raise ValueError(f"{name}: a contiguous buffer of {n} bytes is needed")
        return _dptr(t)

    def _check(self, st: int, allow=()):
        if st != MF_OK and st not in allow:
            raise MFError(st, self.lib.mf_last_error(self.h).decode())
        return st

    def state_tensor(self):
        import torch
        shape = (self.ny, self.nx) if self.dim == 2 else (3, self.nz, self.ny, self.nx)
        return torch.zeros(shape, dtype=torch.float64, device=self.device)

    # -- the C entry points ------------------------------------------------------------------
    def mf_rhs(self, t: float, y, ydot, force_iters: int = 0, seg: int = -2, allow_noconv=False):
        it = ctypes.c_int(0)
        st = self.lib.mf_rhs_ex(self.h, t, seg, self._f64(y, self.state_len, "y"),
                                self._f64(ydot, self.state_len, "ydot"), force_iters, ctypes.byref(it))
        self._check(st, allow=(MF_ERR_NOCONV,) if allow_noconv else ())
        return it.value, st

    def mf_reset_warm(self):
        self._check(self.lib.mf_reset_warm(self.h))

    def mf_set_barrier_timeout(self, seconds: float):
        """Time limit of one grid-barrier wait (<= 0: the default 4 s)."""
        self._check(self.lib.mf_set_barrier_timeout(self.h, float(seconds)))

    def mf_set_state(self, t: float, y=None, h: float = 0.0):
        self._check(self.lib.mf_set_state(self.h, t, h, self._f64(y, self.state_len, "y")))

    def mf_get_state(self, y=None):
        t, h = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.mf_get_state(self.h, ctypes.byref(t), ctypes.byref(h),
                                          self._f64(y, self.state_len, "y")))
        return t.value, h.value

    def mf_advance(self, t_target: float, max_attempts: int = 1 << 40):
        return self._check(self.lib.mf_advance(self.h, t_target, max_attempts))

    def mf_step(self, t_max: float) -> bool:
        acc = ctypes.c_int(0)
        self._check(self.lib.mf_step(self.h, t_max, ctypes.byref(acc)))
        return bool(acc.value)

    def mf_run_ramp(self, t_out, want_fields: bool = False):
        import torch
        t_out = np.ascontiguousarray(t_out, dtype=np.float64)
        nm = 1 if self.dim == 2 else 3
        m = np.zeros(len(t_out) * nm)
        fields = None
        if want_fields:
            per = self.nx * self.ny if self.dim == 2 else 3 * self.nx * self.ny * self.nz
            fields = torch.zeros((len(t_out), per), dtype=torch.float64, device=self.device)
        self._check(self.lib.mf_run_ramp(self.h, len(t_out), _arr(t_out, ctypes.c_double),
                                         _arr(m, ctypes.c_double), _dptr(fields)))
        return m.reshape(len(t_out), nm), fields

    def mf_readout(self, what: int, out=None, t=None, y=None):
        if what == MF_READ_MOMENT:
            nm = 1 if self.dim == 2 else 3
            host = np.zeros(nm)
            ptr = ctypes.c_void_p(host.ctypes.data)
            if y is None:
                self._check(self.lib.mf_readout(self.h, what, ptr))
            else:
                self._check(self.lib.mf_readout_of(self.h, what, t, self._f64(y, self.state_len, "y"), ptr))
            return host
        dout = self._f64(out, self._readout_len(what), "out")
        if y is None:
            self._check(self.lib.mf_readout(self.h, what, dout))
        else:
            self._check(self.lib.mf_readout_of(self.h, what, t, self._f64(y, self.state_len, "y"), dout))
        return out

    def mf_get_info(self) -> dict:
        inf = mf_info()
        self._check(self.lib.mf_get_info(self.h, ctypes.byref(inf)))
        return {name: getattr(inf, name) for name, _ in mf_info._fields_}

    def mf_autotune(self, reps: int = 3, force_iters: int = 2) -> dict:
        """Time the accepted work-item shapes and launch widths and keep the fastest."""
        tu = mf_tuning()
        self._check(self.lib.mf_autotune(self.h, reps, force_iters, ctypes.byref(tu)))
        return {name: getattr(tu, name) for name, _ in mf_tuning._fields_}

    def mf_checkpoint_save(self, out=None):
        """Save a checkpoint into `out` (a uint8 tensor of mf_checkpoint_bytes, device or host;
        allocated on the problem's device if None) and return it."""
        import torch
        n = self.lib.mf_checkpoint_bytes(self.h)
        if out is None:
            out = torch.empty(n, dtype=torch.uint8, device=self.device)
        self._check(self.lib.mf_checkpoint_save(self.h, self._blob(out, "out")))
        return out

    def mf_checkpoint_restore(self, blob):
        self._check(self.lib.mf_checkpoint_restore(self.h, self._blob(blob, "blob")))

    def mf_film_outside_vjp(self, v, iters: int, out=None):
        """Cotangents (of h_dot_in as a device tensor, of h_e_dot as a float) of the film's
        cold-started, fixed-count outside iteration for the cotangent v of its output."""
        import torch
        if out is None:
            out = torch.empty_like(v)
        sb = ctypes.c_double(0.0)
        n = self.state_len
        self._check(self.lib.mf_film_outside_vjp(self.h, iters, self._f64(v, n, "v"), self._f64(out, n, "out"),
                                                 ctypes.byref(sb)))
        return out, sb.value

    def mf_film_rhs_vjp(self, g, v, iters: int):
        """Cotangents (of g and of the jc map as device tensors, of h_e_dot as a float) of the
        film right-hand side with a cold-started, fixed-count outside iteration."""
        import torch
        gbar, jcbar = torch.empty_like(v), torch.empty_like(v)
        sb = ctypes.c_double(0.0)
        n = self.state_len
        self._check(self.lib.mf_film_rhs_vjp(self.h, iters, self._f64(g, n, "g"), self._f64(v, n, "v"),
                                             self._f64(gbar, n, "gbar"), self._f64(jcbar, n, "jcbar"),
                                             ctypes.byref(sb)))
        return gbar, jcbar, sb.value

    def mf_film_rhs_vjp_warm(self, g, v, iters: int, wbar_out=None):
        """Cotangents (of g, of the jc map, of the warm start as device tensors, of h_e_dot as a
        float) of one warm-started film right-hand side with `iters` outside iterations."""
        import torch
        gbar, jcbar, wbar = torch.empty_like(v), torch.empty_like(v), torch.empty_like(v)
        sb = ctypes.c_double(0.0)
        n = self.state_len
        self._check(self.lib.mf_film_rhs_vjp_warm(self.h, iters, self._f64(g, n, "g"), self._f64(v, n, "v"),
                                                  self._f64(wbar_out, n, "wbar_out"),
                                                  self._f64(gbar, n, "gbar"), self._f64(jcbar, n, "jcbar"),
                                                  self._f64(wbar, n, "wbar"), ctypes.byref(sb)))
        return gbar, jcbar, wbar, sb.value

    def mf_film_solve_gradient(self, g0, target, steps, iters, ckpt_every: int = 20, warm0=None,
                               grad: bool = True, warm0_grad: bool = False, hz_out=None):
        """Loss of the frozen-step, frozen-count solve over steps = [(t, h), ...] with
        iters = 3 outside-iteration counts per step; with grad, also dL/djc (device tensor),
        dL/d(knot values) (list) and, with warm0_grad, dL/dwarm0 (device tensor); hz_out (a device
        tensor of the grid, optional) receives h_z(T) of the forward.
        Returns (loss, jcbar, knots_bar, warm0_bar) (None where not computed)."""
        import torch
        n = len(steps)
        iters = [int(i) for i in iters]
        if len(iters) != 3 * n:
            raise ValueError(f"iters needs 3 counts per step ({3 * n}), got {len(iters)}")
        K = self.params.he_knots
        ts = (ctypes.c_double * n)(*[float(t) for t, _ in steps])
        hs = (ctypes.c_double * n)(*[float(h) for _, h in steps])
        it = (ctypes.c_int * (3 * n))(*iters)
        nb = self.lib.mf_film_solve_gradient_work_bytes(self.h, n, ckpt_every)
        work = torch.empty(nb, dtype=torch.uint8, device=self.device)
        jcbar = torch.empty_like(g0) if grad else None
        kb = (ctypes.c_double * max(K, 1))() if grad else None
        wb = torch.empty_like(g0) if (grad and warm0_grad) else None
        loss = ctypes.c_double(0.0)
        m = self.state_len
        self._check(self.lib.mf_film_solve_gradient(
            self.h, n, ts, hs, it, ckpt_every, self._f64(g0, m, "g0"), self._f64(warm0, m, "warm0"),
            self._f64(target, m, "target"), _dptr(work), nb, self._f64(jcbar, m, "jcbar"), kb,
            K if grad else 0, self._f64(wb, m, "warm0_bar"), self._f64(hz_out, m, "hz_out"),
            ctypes.byref(loss)))
        return loss.value, jcbar, (list(kb)[:K] if grad else None), wb

    def mf_set_jc_map(self, jc):
        """jc: device float64 tensor of the grid's cells."""
        self._check(self.lib.mf_set_jc_map(self.h, self._f64(jc, self.nx * self.ny * self.nz, "jc")))

    def mf_set_knot_values(self, values):
        v = [float(x) for x in values]
        if len(v) != self.params.he_knots:
            raise ValueError(f"the problem has {self.params.he_knots} knots, got {len(v)} values")
        self._check(self.lib.mf_set_knot_values(self.h, (ctypes.c_double * len(v))(*v), len(v)))

    def mf_get_log(self, cap: int = 1 << 16):
        buf = (mf_step_log * cap)()
        cnt = ctypes.c_longlong(0)
        self._check(self.lib.mf_get_log(self.h, buf, cap, ctypes.byref(cnt)))
        n = min(cnt.value, cap)
        return [(e.t, e.h, e.t_new, e.outcome, tuple(e.iters), e.err) for e in buf[:n]]

    def close(self):
        if getattr(self, "h", None):
            self.lib.mf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mf_film_rhs_noalloc(problem: "Problem", t: float, y, ydot, force_iters: int = 0,
                        stream=None):
    """Film right-hand side through the entry point that allocates nothing (static scratch).

    For callers that cannot allocate device memory; uses the parameters of `problem` but not
    its workspace or warm start.  Returns (status, iterations, message)."""
    lib = load()
    it = ctypes.c_int(0)
    msg = ctypes.create_string_buffer(256)
    s = stream if stream is not None else problem.stream
    n = problem.state_len
    st = lib.mf_film_rhs_noalloc(ctypes.byref(problem.params), t, problem._f64(y, n, "y"),
                                 problem._f64(ydot, n, "ydot"),
                                 force_iters, ctypes.c_void_p(s.cuda_stream), ctypes.byref(it),
                                 msg, 256)
    return st, it.value, msg.value.decode()


def batch_plan(nx, ny, own_grid, coresident: int, work=None):
    """mf_batch_plan (host only): (number of shared launches, order, launch, ctas)."""
    lib = load()
    n = len(nx)
    arr = lambda v: (ctypes.c_int * max(n, 1))(*[int(x) for x in v])
    order, launch, ctas = arr([0] * n), arr([0] * n), arr([0] * n)
    w = None if work is None else (ctypes.c_double * max(n, 1))(*[float(x) for x in work])
    r = lib.mf_batch_plan(n, arr(nx), arr(ny), arr(own_grid), w, int(coresident), order, launch, ctas)
    if r < 0:
        raise ValueError("mf_batch_plan: invalid arguments")
    return r, list(order)[:n], list(launch)[:n], list(ctas)[:n]


def advance_batch(problems, t_targets, max_attempts: int = 1 << 40):
    """mf_advance_batch: advance several problems together (films of one precision in shared
    persistent launches, bulk bodies one launch each).  Returns the list of per-problem status
    codes; raises on the first failure like the single-problem calls."""
    lib = load()
    n = len(problems)
    hs = (ctypes.c_void_p * n)(*[p.h for p in problems])
    ts = (ctypes.c_double * n)(*[float(t) for t in t_targets])
    st = (ctypes.c_int * n)()
    r = lib.mf_advance_batch(hs, n, ts, max_attempts, st)
    out = list(st)
    if r != 0:
        bad = next((i for i, v in enumerate(out) if v != 0), None)
        if bad is None:          # refused before any problem ran
            raise MFError(r, "mf_advance_batch refused its arguments (a NULL or repeated problem)")
        raise MFError(r, f"problem {bad}: " + lib.mf_last_error(problems[bad].h).decode())
    return out


def from_workload(wl, **over) -> Problem:
    """Problem for a workloads.Workload description."""
    kw = dict(dim=wl.dim, nx=wl.nx, ny=wl.ny, nz=wl.nz, Lx=wl.Lx, Ly=wl.Ly, Lz=wl.Lz,
              mask=wl.mask, n=wl.n, rho_out=wl.rho_out, precision=wl.precision,
              jc=wl.jc, jc_map=wl.jc_map, sigma=wl.sigma, lam=wl.lam, iter_tol=wl.iter_tol,
              iter_max=wl.iter_max, rtol=wl.rtol, atol=wl.atol, he_knots=wl.he_knots,
              he_sin=wl.he_sin, he_dir=wl.vector_he, gamma=getattr(wl, "gamma", 1.0),
              b0=getattr(wl, "b0", 0.0))
    kw.update(over)
    return Problem(**kw)
