"""Thin ctypes binding of libtgms (include/tgms.h): same entry-point names,
argument marshalling only.  Every step of the solver runs in the library's
CUDA kernels; nothing here computes.

Device arrays are passed as torch CUDA tensors (float64, contiguous) through
their data pointers; host arrays (TG_PTR_HOST mode) as C-contiguous float64
numpy arrays.  The library must have been built (``build.build_library``);
``lib()`` raises if it is missing -- there is no fallback.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libtgms.so")

TG_OK = 0
ERRORS = {
    -1: "TG_ERR_INVALID_ARG", -2: "TG_ERR_INCOMPATIBLE_SOURCE", -3: "TG_ERR_BREAKDOWN",
    -4: "TG_ERR_MAXITER", -5: "TG_ERR_DEVICE_TIMEOUT", -6: "TG_ERR_CUDA", -7: "TG_ERR_OOM",
    -8: "TG_ERR_UNSUPPORTED", -9: "TG_ERR_DEGENERATE_BASIS",
}
PREC = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
COARSE = {"gmsfem": 0, "msfem": 1, "rt0": 2, "learned": 3}
CYCLE = {"two_grid": 0, "additive": 1}
COARSE_SOLVER = {"auto": 0, "dense": 1, "nd": 2}
PTR_HOST, PTR_DEVICE = 0, 1

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
c_int_p, c_double_p = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)


class tg_grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("bx", c_int), ("by", c_int), ("overlap", c_int)]


class tg_options(ctypes.Structure):
    _fields_ = [("eta", c_double), ("m1", c_int), ("m2", c_int), ("precision", c_int),
                ("flexible", c_int), ("max_iter", c_int), ("pointer_mode", c_int),
                ("coarse_space", c_int), ("max_basis", c_int), ("profile", c_int),
                ("net", c_void_p), ("face_profiles", c_void_p), ("learned_k", c_int),
                ("learned_max_iter", c_int), ("smoother_shape", c_int), ("launch_overlap", c_int),
                ("cycle", c_int), ("batch_lockstep", c_int), ("batch_nets", c_void_p), ("batch_nnets", c_int),
                ("coarse_solver", c_int)]


class tg_report(ctypes.Structure):
    _fields_ = [("iters", c_int), ("converged", c_int), ("rel_residual", c_double),
                ("cond_estimate", c_double), ("coarse_dim", c_int), ("velocity_basis", c_int),
                ("coarse_unknowns", c_int), ("max_div_error", c_double),
                ("preprocess_ms", c_double), ("pcg_ms", c_double), ("epilogue_ms", c_double),
                ("kernel_launches", c_int), ("smoother_launches", c_int), ("smoother_ms", c_double),
                ("graph", c_int), ("snapshot_solves", c_int), ("fallback_faces", c_int),
                ("learned_fallback", c_int), ("smoother_shape", c_int), ("shape_us", ctypes.c_float * 10),
                ("refactored_patches", c_int), ("refactored_blocks", c_int),
                ("update_rank", c_int * 2), ("operator_launches", c_int), ("operator_ms", c_double),
                ("coarse_solver", c_int), ("coarse_solve_mb", c_double)]

    def shape_times(self):
        return [float(v) for v in self.shape_us]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class TgmsError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.tg_strerror(code).decode() if _lib is not None else ""
        super().__init__("%s failed: %s (%s)" % (where, ERRORS.get(code, code), msg))


_lib = None

# name -> (restype, argtypes)
SIGNATURES = {
    "tg_default_options": (c_int, [ctypes.POINTER(tg_options)]),
    "tg_setup": (c_int, [c_void_p, ctypes.POINTER(tg_grid), c_double, ctypes.POINTER(tg_options),
                         c_void_p, ctypes.POINTER(c_void_p)]),
    "tg_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p,
                         c_int_p, ctypes.POINTER(tg_report)]),
    "tg_destroy": (None, [c_void_p]),
    "tg_update_kappa": (c_int, [c_void_p, c_void_p, c_int]),
    "tg_total_mobility": (c_int, [c_void_p, c_void_p, c_int, c_double, c_double, c_void_p, c_void_p]),
    "tg_transport_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double, c_double, c_double,
                                  c_double, c_void_p, c_double_p, c_void_p]),
    "tg_solve_warm": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_int_p, ctypes.POINTER(tg_report)]),
    "tg_strerror": (ctypes.c_char_p, [c_int]),
    "tg_probe_bounded_wait": (c_int, [c_int, c_int, c_void_p]),
    "tg_apply_operator": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "tg_apply_smoother": (c_int, [c_void_p, c_void_p, c_void_p]),
    "tg_apply_coarse": (c_int, [c_void_p, c_void_p, c_void_p]),
    "tg_apply_preconditioner": (c_int, [c_void_p, c_void_p, c_void_p]),
    "tg_coarse_info": (c_int, [c_void_p, c_int_p, c_int_p, c_void_p, c_void_p]),
    "tg_preprocess": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "tg_pressure_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "tg_setup_batch": (c_int, [c_int, c_void_p, c_void_p, c_double, ctypes.POINTER(tg_options), c_int, c_void_p,
                               ctypes.POINTER(c_void_p)]),
    "tg_solve_batch": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p]),
    "tg_batch_size": (c_int, [c_void_p, c_int_p, c_int_p]),
    "tg_destroy_batch": (None, [c_void_p]),
    "tg_mlp_shape": (c_int, [c_int, c_int, c_int, c_int_p, c_int_p, ctypes.POINTER(ctypes.c_longlong)]),
    "tg_mlp_create": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, ctypes.POINTER(c_void_p)]),
    "tg_mlp_params": (c_int, [c_void_p, c_void_p]),
    "tg_mlp_forward": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "tg_mlp_loss_grad": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double_p, c_void_p]),
    "tg_mlp_train": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_int, ctypes.c_float,
                             c_void_p]),
    "tg_mlp_destroy": (None, [c_void_p]),
    "tg_face_data": (c_int, [c_void_p, ctypes.POINTER(tg_grid), c_double, c_int, c_void_p, c_void_p, c_void_p,
                             c_void_p, c_void_p]),
}


def lib():
    """Load libtgms.so from the package tree (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtgms.so not built: run paper_1807_07220_gb300.build.build_library()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    """Data pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, where):
    if rc != TG_OK:
        raise TgmsError(rc, where)


def default_options(**kw):
    """tg_default_options plus overrides; ``net`` takes an Mlp (or a raw
    handle), ``face_profiles`` a device tensor."""
    o = tg_options()
    _check(lib().tg_default_options(ctypes.byref(o)), "tg_default_options")
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PREC[v]
        if k == "coarse_space" and isinstance(v, str):
            v = COARSE[v]
        if k == "cycle" and isinstance(v, str):
            v = CYCLE[v]
        if k == "coarse_solver" and isinstance(v, str):
            v = COARSE_SOLVER[v]
        if k == "net":
            v = getattr(v, "handle", v)
            v = v.value if isinstance(v, ctypes.c_void_p) else v
        if k == "face_profiles":
            v = _ptr(v).value if v is not None else None
        if k == "batch_nets":
            # a host array of network handles, kept alive with the options
            hs = [getattr(x, "handle", x) for x in v]
            arr = (c_void_p * len(hs))(*[x.value if isinstance(x, ctypes.c_void_p) else x for x in hs])
            o._batch_nets_keep = arr
            o.batch_nnets = len(hs)
            v = ctypes.cast(arr, c_void_p).value
        setattr(o, k, v)
    return o


def tg_setup(kappa, n, b, eig_tol, overlap=2, options=None, stream=0):
    """Returns an opaque handle (c_void_p).  kappa: n*n float64 (device tensor
    or host array per options.pointer_mode)."""
    g = tg_grid(n, n, b, b, overlap)
    o = options if options is not None else default_options()
    h = ctypes.c_void_p()
    _check(lib().tg_setup(_ptr(kappa), ctypes.byref(g), float(eig_tol), ctypes.byref(o),
                          ctypes.c_void_p(stream), ctypes.byref(h)), "tg_setup")
    return h


def tg_solve(h, f, bflux, rtol, ux, uy, p, allow_maxiter=False):
    it = ctypes.c_int(0)
    rep = tg_report()
    rc = lib().tg_solve(h, _ptr(f), _ptr(bflux), float(rtol), _ptr(ux), _ptr(uy), _ptr(p),
                        ctypes.byref(it), ctypes.byref(rep))
    if not (allow_maxiter and rc == -4):
        _check(rc, "tg_solve")
    return it.value, rep


def tg_solve_warm(h, f, bflux, rtol, ux0, uy0, ux, uy, p, allow_maxiter=False):
    it = ctypes.c_int(0)
    rep = tg_report()
    rc = lib().tg_solve_warm(h, _ptr(f), _ptr(bflux), float(rtol), _ptr(ux0), _ptr(uy0), _ptr(ux), _ptr(uy),
                             _ptr(p), ctypes.byref(it), ctypes.byref(rep))
    if not (allow_maxiter and rc == -4):
        _check(rc, "tg_solve_warm")
    return it.value, rep


def tg_update_kappa(h, kappa, coarse=0):
    _check(lib().tg_update_kappa(h, _ptr(kappa), int(coarse)), "tg_update_kappa")


def tg_total_mobility(kappa, s, n, mu_w, mu_o, out, stream=0):
    _check(lib().tg_total_mobility(_ptr(kappa), _ptr(s), int(n), float(mu_w), float(mu_o), _ptr(out),
                                   ctypes.c_void_p(stream)), "tg_total_mobility")


def tg_transport_step(s, ux, uy, f, n, cfl, mu_w, mu_o, s_out, dt_fixed=0.0, stream=0):
    """Returns the time step taken."""
    dt = ctypes.c_double(0.0)
    _check(lib().tg_transport_step(_ptr(s), _ptr(ux), _ptr(uy), _ptr(f), int(n), float(cfl), float(dt_fixed),
                                   float(mu_w), float(mu_o), _ptr(s_out), ctypes.byref(dt),
                                   ctypes.c_void_p(stream)), "tg_transport_step")
    return dt.value


def tg_destroy(h):
    if h is not None:
        lib().tg_destroy(h)


def tg_probe_bounded_wait(complete, limit_log2, stream=0):
    """TG_OK (0) or TG_ERR_DEVICE_TIMEOUT (-5): see include/tgms.h."""
    return lib().tg_probe_bounded_wait(int(complete), int(limit_log2), ctypes.c_void_p(stream))


def tg_strerror(code):
    return lib().tg_strerror(code).decode()


def tg_apply_operator(h, psi, out, precision=0):
    _check(lib().tg_apply_operator(h, _ptr(psi), _ptr(out), int(precision)), "tg_apply_operator")


def tg_apply_smoother(h, rho, z):
    _check(lib().tg_apply_smoother(h, _ptr(rho), _ptr(z)), "tg_apply_smoother")


def tg_apply_coarse(h, rho, z):
    _check(lib().tg_apply_coarse(h, _ptr(rho), _ptr(z)), "tg_apply_coarse")


def tg_apply_preconditioner(h, rho, z):
    _check(lib().tg_apply_preconditioner(h, _ptr(rho), _ptr(z)), "tg_apply_preconditioner")


def tg_coarse_info(h, b):
    """Returns (nsel per face, eigenvalues (nfaces, b), velocity basis count)."""
    import numpy as np
    nf, vb = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().tg_coarse_info(h, ctypes.byref(nf), ctypes.byref(vb), None, None), "tg_coarse_info")
    nsel = np.zeros(nf.value, dtype=np.int32)
    lam = np.zeros((nf.value, b), dtype=np.float64)
    _check(lib().tg_coarse_info(h, None, None, _ptr(nsel), _ptr(lam)), "tg_coarse_info")
    return nsel, lam, vb.value


def tg_preprocess(h, f, bflux, ux, uy):
    _check(lib().tg_preprocess(h, _ptr(f), _ptr(bflux), _ptr(ux), _ptr(uy)), "tg_preprocess")


def _ptr_array(arrs):
    """C array of data pointers (None entries -> NULL)."""
    arr = (c_void_p * len(arrs))()
    for k, a in enumerate(arrs):
        arr[k] = None if a is None else _ptr(a).value
    return arr


def tg_setup_batch(kappas, ns, bs, eig_tol, nrhs, overlap=2, options=None, stream=0):
    """kappas: list of device tensors (n_i, n_i); returns an opaque batch handle."""
    ninst = len(kappas)
    grids = (tg_grid * ninst)(*[tg_grid(n, n, b, b, overlap) for n, b in zip(ns, bs)])
    o = options if options is not None else default_options()
    h = ctypes.c_void_p()
    _check(lib().tg_setup_batch(ninst, _ptr_array(kappas), grids, float(eig_tol), ctypes.byref(o), int(nrhs),
                                ctypes.c_void_p(stream), ctypes.byref(h)), "tg_setup_batch")
    return h


def tg_solve_batch(batch, f, bflux, rtol, ux, uy, p, allow_maxiter=False):
    """Lists of device tensors (instance-major, nrhs per instance); bflux may be None.
    Returns (iterations, status codes) per problem."""
    import numpy as np
    m = len(f)
    iters = np.zeros(m, dtype=np.int32)
    status = np.zeros(m, dtype=np.int32)
    rc = lib().tg_solve_batch(batch, _ptr_array(f), None if bflux is None else _ptr_array(bflux), float(rtol),
                              _ptr_array(ux), _ptr_array(uy), _ptr_array(p), _ptr(iters), _ptr(status))
    if not (allow_maxiter and rc == -4):
        _check(rc, "tg_solve_batch")
    return iters, status


def tg_destroy_batch(batch):
    if batch is not None:
        lib().tg_destroy_batch(batch)


def tg_batch_size(batch):
    ni, nr = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().tg_batch_size(batch, ctypes.byref(ni), ctypes.byref(nr)), "tg_batch_size")
    return ni.value, nr.value


def tg_pressure_noalloc(kappa, ux, uy, p, n, stream=0):
    """Allocation-free pressure recovery (device tensors; see include/tgms.h)."""
    _check(lib().tg_pressure_noalloc(_ptr(kappa), _ptr(ux), _ptr(uy), _ptr(p), int(n),
                                     ctypes.c_void_p(stream)), "tg_pressure_noalloc")


# ---------------------------------------------------------------- learned coarse basis
def tg_mlp_shape(b, k, hidden):
    din, dout, npar = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_longlong(0)
    _check(lib().tg_mlp_shape(int(b), int(k), int(hidden), ctypes.byref(din), ctypes.byref(dout),
                              ctypes.byref(npar)), "tg_mlp_shape")
    return din.value, dout.value, npar.value


class Mlp:
    """Owner of a tg_mlp handle.  Tensors are torch CUDA tensors: parameters
    float32, inputs bfloat16 (passed as uint16 bit patterns), labels float32."""

    def __init__(self, b, k, hidden, params, stream=0):
        self.b, self.k, self.hidden = b, k, hidden
        self.din, self.dout, self.nparam = tg_mlp_shape(b, k, hidden)
        if params.numel() != self.nparam:
            raise ValueError("parameter vector has %d entries, expected %d" % (params.numel(), self.nparam))
        self.handle = ctypes.c_void_p()
        _check(lib().tg_mlp_create(b, k, hidden, _ptr(params), ctypes.c_void_p(stream),
                                   ctypes.byref(self.handle)), "tg_mlp_create")

    def params(self, out):
        _check(lib().tg_mlp_params(self.handle, _ptr(out)), "tg_mlp_params")
        return out

    def forward(self, x, y):
        _check(lib().tg_mlp_forward(self.handle, int(x.shape[0]), _ptr(x), _ptr(y)), "tg_mlp_forward")
        return y

    def loss_grad(self, x, q, grad=None):
        loss = ctypes.c_double(0.0)
        _check(lib().tg_mlp_loss_grad(self.handle, int(x.shape[0]), _ptr(x), _ptr(q), ctypes.byref(loss),
                                      _ptr(grad)), "tg_mlp_loss_grad")
        return loss.value

    def train(self, x, q, order, nsteps, batch, lr, loss_hist=None):
        _check(lib().tg_mlp_train(self.handle, int(x.shape[0]), _ptr(x), _ptr(q), _ptr(order), int(nsteps),
                                  int(batch), float(lr), _ptr(loss_hist)), "tg_mlp_train")

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().tg_mlp_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tg_face_data(kappa, n, b, eig_tol, k, x, q, nsel=None, lam=None, overlap=2, stream=0):
    """Training data of one field (device tensors): x (faces x din, uint16 =
    bfloat16 bits), q (faces x k x b float32), nsel (faces int32), lam
    (faces x b float64)."""
    g = tg_grid(n, n, b, b, overlap)
    _check(lib().tg_face_data(_ptr(kappa), ctypes.byref(g), float(eig_tol), int(k), ctypes.c_void_p(stream),
                              _ptr(x), _ptr(q), _ptr(nsel), _ptr(lam)), "tg_face_data")


class Solver:
    """Convenience owner of a handle plus output buffers on one CUDA device.

    Inputs and outputs are torch float64 CUDA tensors; arrays are (n, n)
    [j, i], ux (n, n+1), uy (n+1, n)."""

    def __init__(self, kappa, b, eig_tol, overlap=2, device="cuda", stream=None, **opts):
        import torch
        if opts.get("pointer_mode", PTR_DEVICE) != PTR_DEVICE:
            raise ValueError("Solver passes device tensors; use tg_setup/tg_solve for host pointers")
        self.torch = torch
        n = kappa.shape[0]
        self.n, self.b = n, b
        self.device = torch.device(device)
        self.kappa = torch.as_tensor(kappa, dtype=torch.float64, device=self.device).contiguous()
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = tg_setup(self.kappa, n, b, eig_tol, overlap, default_options(**opts),
                          self.stream.cuda_stream)
        z = lambda *s: torch.zeros(*s, dtype=torch.float64, device=self.device)
        self.ux, self.uy, self.p = z(n, n + 1), z(n + 1, n), z(n, n)

    def solve(self, f, bflux=None, rtol=1e-8, allow_maxiter=False, ux0=None):
        """ux0: optional initial guess of the x-face velocities (tg_solve_warm)."""
        t = self.torch
        f = t.as_tensor(f, dtype=t.float64, device=self.device).contiguous()
        bf = None if bflux is None else t.as_tensor(bflux, dtype=t.float64, device=self.device).contiguous()
        if ux0 is not None:
            u0 = t.as_tensor(ux0, dtype=t.float64, device=self.device).contiguous()
            return tg_solve_warm(self.h, f, bf, rtol, u0, None, self.ux, self.uy, self.p, allow_maxiter)
        it, rep = tg_solve(self.h, f, bf, rtol, self.ux, self.uy, self.p, allow_maxiter)
        return it, rep

    def close(self):
        if self.h is not None:
            tg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
