"""Python binding of librhi, the GB300 implicit radiation / ionization / gas-energy step.

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.  The
functions keep the C names of ``include/rhi.h``; ``Solver`` wraps one handle.  Importing this
package does not load the library; the first call does, and fails loudly when ``librhi.so``
has not been built (``paper_0901_1110_gb300._build.build()``).
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librhi.so")

RHI_OK, RHI_ERR_ARG, RHI_ERR_CUDA, RHI_ERR_NONCONVERGED, RHI_ERR_NONPHYSICAL, RHI_ERR_STATE = range(6)
RHI_BC_ZERO_FLUX, RHI_BC_PERIODIC, RHI_BC_DIRICHLET = 0, 1, 2
RHI_GUESS_PREVIOUS, RHI_GUESS_PREDICTOR, RHI_GUESS_LEARNED = 0, 1, 2
RHI_PRECOND_JACOBI, RHI_PRECOND_MG_FP64, RHI_PRECOND_MG_FP32 = 0, 1, 2
RHI_SPECTRUM_MONO, RHI_SPECTRUM_BLACKBODY, RHI_SPECTRUM_POWERLAW = 0, 1, 2
RHI_MODEL_IONIZATION, RHI_MODEL_LTE = 0, 1


class rhi_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double)]


class rhi_bc(C.Structure):
    _fields_ = [("kind", C.c_int * 6), ("value", C.c_double * 6)]


class rhi_params(C.Structure):
    _fields_ = [("n_species", C.c_int), ("y_he", C.c_double), ("theta", C.c_double),
                ("m_grey", C.c_int), ("isothermal", C.c_int), ("limiter", C.c_int),
                ("kappa_floor", C.c_double), ("u_e", C.c_double), ("u_n", C.c_double),
                ("u_E", C.c_double), ("tau", C.c_double), ("lam_min", C.c_double),
                ("mlp_gate", C.c_double), ("mlp_ood", C.c_double), ("mlp_restart", C.c_int), ("mlp_retry", C.c_int), ("growth_max", C.c_double), ("watchdog", C.c_int), ("limiter_jacobian", C.c_int),
                ("max_newton", C.c_int), ("max_pcg", C.c_int), ("guess", C.c_int),
                ("precond", C.c_int), ("mg_levels", C.c_int), ("mg_pre", C.c_int),
                ("mg_post", C.c_int), ("mg_coarse_sweeps", C.c_int), ("mg_omega", C.c_double), ("vcycle_graph", C.c_int),
                ("krylov_graph", C.c_int), ("mg_matrix", C.c_int), ("predict_final", C.c_int),
                ("krylov_restart", C.c_double),
                ("dt_norm", C.c_int), ("dt_tau_tol", C.c_double), ("model", C.c_int),
                ("kappa_total", C.c_double), ("kappa_planck", C.c_double), ("mu", C.c_double),
                ("sk", C.c_double * 3), ("pgam", C.c_double * 3), ("ph", C.c_double * 3),
                ("photon_energy", C.c_double)]


class rhi_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_its", C.c_int), ("pcg_its", C.c_int),
                ("vcycles", C.c_int), ("backtracks", C.c_int), ("lam_min_steps", C.c_int),
                ("guess_used", C.c_int), ("launches", C.c_int), ("guess_restarts", C.c_int), ("krylov_fallbacks", C.c_int), ("host_syncs", C.c_int), ("krylov_stalls", C.c_int),
                ("final_predicted", C.c_int), ("final_missed", C.c_int),
                ("res_initial", C.c_double),
                ("res_final", C.c_double), ("res_guess_prev", C.c_double), ("ms", C.c_double),
                ("eps_loc", C.c_double), ("dt_next", C.c_double),
                ("res_history", C.c_double * 64)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "rhi_params_default": (C.c_int, [C.POINTER(rhi_params), C.c_int]),
    "rhi_grey_constants": (C.c_int, [C.c_int, C.c_double, C.c_int, _D, _D, _D, _D]),
    "rhi_create": (C.c_int, [C.POINTER(rhi_grid), C.POINTER(rhi_bc), C.POINTER(rhi_params), _P,
                             C.POINTER(_P)]),
    "rhi_set_state": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int]),
    "rhi_set_sources": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), _D]),
    "rhi_implicit_step": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_double]),
    "rhi_get_state": (C.c_int, [_P, _P, _P, _P, C.c_int]),
    "rhi_get_stats": (C.c_int, [_P, C.POINTER(rhi_stats)]),
    "rhi_linearize": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, _P, _P, _P, _P, _P,
                                C.c_int]),
    "rhi_precond_apply": (C.c_int, [_P, _P, _P, C.c_int]),
    "rhi_residual": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, _P, _P, _D, C.c_int]),
    "rhi_mlp_guess": (C.c_int, [_P, C.c_double, C.c_double, _P, C.c_int]),
    "rhi_set_profiling": (C.c_int, [_P, C.c_int]),
    "rhi_set_profiling_names": (C.c_int, [_P, C.c_char_p]),
    "rhi_kernel_times": (C.c_int, [_P, C.c_int, C.c_char_p, _D, C.POINTER(C.c_int)]),
    "rhi_rms_norm_noalloc": (C.c_int, [_P, C.c_longlong, C.c_longlong, _P, _P]),
    "rhi_advance": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                              C.c_double, C.c_double, C.c_double, C.c_int, _D,
                              C.POINTER(C.c_int)]),
    "rhi_mlp_set_weights": (C.c_int, [_P, _P, C.c_size_t]),
    "rhi_mlp_get_weights": (C.c_int, [_P, _P, C.c_size_t]),
    "rhi_mlp_features": (C.c_int, [_P, C.c_double, C.c_double, _P, C.c_int]),
    "rhi_mlp_targets": (C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
    "rhi_mlp_forward": (C.c_int, [_P, _P, _P, C.c_longlong, C.c_int]),
    "rhi_mlp_loss_grad": (C.c_int, [_P, _P, _P, C.c_longlong, _P, _D, C.c_int]),
    "rhi_mlp_train": (C.c_int, [_P, _P, _P, C.c_longlong, C.c_int, C.c_int, C.c_double, _D]),
    "rhi_last_error": (C.c_char_p, [_P]),
    "rhi_status_string": (C.c_char_p, [C.c_int]),
    "rhi_destroy": (None, [_P]),
}

_lib = None


def lib():
    """The loaded librhi.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_0901_1110_gb300._build.build() (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class RhiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


# ---- C functions under their own names ---------------------------------------------------------

def rhi_params_default(n_species):
    p = rhi_params()
    rc = lib().rhi_params_default(C.byref(p), n_species)
    if rc:
        raise RhiError(rc, "rhi_params_default")
    return p


def rhi_grey_constants(spectrum, param, n_species):
    sk, pg, ph = (C.c_double * 3)(), (C.c_double * 3)(), (C.c_double * 3)()
    eps = C.c_double()
    rc = lib().rhi_grey_constants(spectrum, param, n_species, sk, pg, ph, C.byref(eps))
    if rc:
        raise RhiError(rc, "rhi_grey_constants")
    return dict(sk=np.array(sk[:]), pgam=np.array(pg[:]), ph=np.array(ph[:]), eps=eps.value)


RHI_NOALLOC_MAX_COUNT = 33554432
RHI_MLP_IN, RHI_MLP_HID, RHI_MLP_OUT = 13, 64, 6
RHI_MLP_NWEIGHTS = (RHI_MLP_HID * RHI_MLP_IN + RHI_MLP_HID + 2 * (RHI_MLP_HID * RHI_MLP_HID + RHI_MLP_HID)
                    + RHI_MLP_OUT * RHI_MLP_HID + RHI_MLP_OUT + 2 * RHI_MLP_IN)


def rhi_rms_norm_noalloc(v_ptr, n, count, out_ptr, stream=None):
    """Allocation-free RMS norm of n doubles at device address v_ptr into the device double at
    out_ptr (enqueued on `stream`); returns the status code."""
    return lib().rhi_rms_norm_noalloc(v_ptr, n, count, out_ptr, stream)


def rhi_status_string(code):
    return lib().rhi_status_string(code).decode()


def _fptr(a, count=None):
    """(pointer, on_device) of a float32 numpy array or tensor, C-contiguous."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be C-contiguous float32")
        ptr, dev = a.ctypes.data, 0
    else:
        if str(a.dtype) != "torch.float32" or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float32")
        ptr, dev = a.data_ptr(), (1 if a.is_cuda else 0)
    if count is not None and (a.size if isinstance(a, np.ndarray) else a.numel()) < count:
        raise ValueError("buffer too small")
    return ptr, dev


def _ptr(a):
    """(pointer, on_device) of a numpy array or a CUDA tensor (float64, contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    # torch tensor
    if a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
        raise TypeError("tensors must be contiguous float64")
    return a.data_ptr(), (1 if a.is_cuda else 0)


class Solver:
    """One rhi handle: grid, boundaries and parameters fixed at creation."""

    def __init__(self, nx, ny, nz, dx, params, bc=(RHI_BC_ZERO_FLUX,) * 6, stream=None,
                 bc_value=(0.0,) * 6):
        self.grid = rhi_grid(nx, ny, nz, dx)
        b = rhi_bc()
        for q in range(6):
            b.kind[q] = int(bc[q])
            b.value[q] = float(bc_value[q])
        self.bc = b
        self.params = params
        self.ns = params.n_species
        self.N = nx * ny * nz
        h = C.c_void_p()
        rc = lib().rhi_create(C.byref(self.grid), C.byref(b), C.byref(params),
                              C.c_void_p(stream or 0), C.byref(h))
        if rc:
            raise RhiError(rc, "rhi_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.rhi_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what, check=True):
        if rc and check:
            raise RhiError(rc, f"{what}: {lib().rhi_last_error(self.h).decode()}")
        return rc

    def set_state(self, E, e, n, nH, src=None):
        (pE, d0), (pe, d1), (pn, d2), (pH, d3) = _ptr(E), _ptr(e), _ptr(n), _ptr(nH)
        ps, d4 = _ptr(src)
        devs = {d0, d1, d3} | ({d2} if n is not None else set()) | ({d4} if src is not None else set())
        if len(devs) != 1:
            raise TypeError("all fields on the host or all on the device")
        return self._check(lib().rhi_set_state(self.h, pE, pe, pn, pH, ps, d0), "rhi_set_state")

    def set_sources(self, ijk, rate):
        ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        rate = np.ascontiguousarray(rate, dtype=np.float64).ravel()
        return self._check(lib().rhi_set_sources(
            self.h, len(rate), ijk.ctypes.data_as(C.POINTER(C.c_int)),
            rate.ctypes.data_as(_D)), "rhi_set_sources")

    def step(self, dt, a=1.0, adot=0.0, newton_tol=1e-8, lin_tol=1e-10, check=True):
        return self._check(lib().rhi_implicit_step(self.h, dt, a, adot, newton_tol, lin_tol),
                           "rhi_implicit_step", check)

    def advance(self, t_end, dt0, dt_min=0.0, dt_max=float("inf"), a=1.0, adot=0.0,
                newton_tol=1e-8, lin_tol=1e-10, max_steps=100000):
        """Adaptive steps (Sec. 3.2.3) until t_end; returns (time reached, steps taken)."""
        t = C.c_double()
        n = C.c_int()
        self._check(lib().rhi_advance(self.h, t_end, dt0, dt_min, dt_max, a, adot, newton_tol,
                                      lin_tol, max_steps, C.byref(t), C.byref(n)), "rhi_advance")
        return t.value, n.value

    def get_state(self, E=None, e=None, n=None):
        """Host copies (numpy) unless device tensors are given to fill."""
        if E is None:
            E = np.empty(self.N)
            e = np.empty(self.N)
            n = np.empty(self.ns * self.N)
        (pE, dev), (pe, _), (pn, _) = _ptr(E), _ptr(e), _ptr(n)
        self._check(lib().rhi_get_state(self.h, pE, pe, pn, dev), "rhi_get_state")
        return dict(E=E, e=e, n=n.reshape(self.ns, self.N) if isinstance(n, np.ndarray) else n)

    def stats(self):
        s = rhi_stats()
        lib().rhi_get_stats(self.h, C.byref(s))
        out = {k: getattr(s, k) for k, _ in rhi_stats._fields_ if k != "res_history"}
        out["res_history"] = list(s.res_history[:min(s.newton_its + 1, 64)])
        return out

    def linearize(self, dt, a=1.0, adot=0.0):
        nv = self.ns + 2
        f = np.empty(nv * self.N)
        d = np.empty(self.N)
        lo = np.empty(3 * self.N)
        hi = np.empty(3 * self.N)
        r = np.empty(self.N)
        self._check(lib().rhi_linearize(self.h, dt, a, adot, f.ctypes.data, d.ctypes.data,
                                        lo.ctypes.data, hi.ctypes.data, r.ctypes.data, 0),
                    "rhi_linearize")
        return dict(f=f.reshape(nv, self.N), diag=d, face=lo.reshape(3, self.N),
                    face_hi=hi.reshape(3, self.N), rhs=r)

    def residual(self, U, dt, a=1.0, adot=0.0):
        """Scaled residual ((ns + 2) x N) and its RMS norm at iterate U = (e_c, n, E)."""
        U = np.ascontiguousarray(U, dtype=np.float64).ravel()
        f = np.empty_like(U)
        nrm = C.c_double()
        self._check(lib().rhi_residual(self.h, dt, a, adot, U.ctypes.data, f.ctypes.data,
                                       C.byref(nrm), 0), "rhi_residual")
        return f.reshape(self.ns + 2, self.N), nrm.value

    def precond_apply(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty_like(r)
        self._check(lib().rhi_precond_apply(self.h, r.ctypes.data, z.ctypes.data, 0),
                    "rhi_precond_apply")
        return z

    # ---- learned guess (an addition to the paper's method) --------------------------------------

    def mlp_set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32).ravel()
        return self._check(lib().rhi_mlp_set_weights(self.h, w.ctypes.data, w.size),
                           "rhi_mlp_set_weights")

    def mlp_get_weights(self):
        w = np.empty(RHI_MLP_NWEIGHTS, dtype=np.float32)
        self._check(lib().rhi_mlp_get_weights(self.h, w.ctypes.data, w.size), "rhi_mlp_get_weights")
        return w

    def mlp_features(self, dt, a=1.0, out=None):
        """Features (N x 13, float32) of the current state; into `out` (array or tensor) if given."""
        X = np.empty((self.N, RHI_MLP_IN), dtype=np.float32) if out is None else out
        pX, dev = _fptr(X, self.N * RHI_MLP_IN)
        self._check(lib().rhi_mlp_features(self.h, dt, a, pX, dev), "rhi_mlp_features")
        return X

    def mlp_targets(self, old, out=None):
        """Targets (N x 6, float32) of the step from `old` (dict E, e, n) to the current state."""
        Y = np.empty((self.N, RHI_MLP_OUT), dtype=np.float32) if out is None else out
        pY, dev = _fptr(Y, self.N * RHI_MLP_OUT)
        (pE, d0), (pe, d1), (pn, d2) = _ptr(old["E"]), _ptr(old["e"]), _ptr(old["n"])
        if len({d0, d1, d2, dev}) != 1:
            raise TypeError("all buffers on the host or all on the device")
        self._check(lib().rhi_mlp_targets(self.h, pE, pe, pn, pY, dev), "rhi_mlp_targets")
        return Y

    def mlp_guess(self, dt, a=1.0):
        """The decoded learned guess (e_c, n, E) as a ((ns + 2) x N) array."""
        U = np.empty((self.ns + 2) * self.N)
        self._check(lib().rhi_mlp_guess(self.h, dt, a, U.ctypes.data, 0), "rhi_mlp_guess")
        return U.reshape(self.ns + 2, self.N)

    def mlp_forward(self, X, out=None):
        n = X.shape[0]
        Y = np.empty((n, RHI_MLP_OUT), dtype=np.float32) if out is None else out
        (pX, d0), (pY, d1) = _fptr(X, n * RHI_MLP_IN), _fptr(Y, n * RHI_MLP_OUT)
        if d0 != d1:
            raise TypeError("X and Y both on the host or both on the device")
        self._check(lib().rhi_mlp_forward(self.h, pX, pY, n, d0), "rhi_mlp_forward")
        return Y

    def mlp_loss_grad(self, X, Y):
        n = X.shape[0]
        (pX, d0), (pY, d1) = _fptr(X, n * RHI_MLP_IN), _fptr(Y, n * RHI_MLP_OUT)
        if d0 != d1:
            raise TypeError("X and Y both on the host or both on the device")
        g = np.empty(RHI_MLP_NWEIGHTS, dtype=np.float32)
        loss = C.c_double()
        if d0:
            import torch
            gd = torch.empty(RHI_MLP_NWEIGHTS, dtype=torch.float32, device=X.device)
            self._check(lib().rhi_mlp_loss_grad(self.h, pX, pY, n, gd.data_ptr(), C.byref(loss), 1),
                        "rhi_mlp_loss_grad")
            g = gd.cpu().numpy()
        else:
            self._check(lib().rhi_mlp_loss_grad(self.h, pX, pY, n, g.ctypes.data, C.byref(loss), 0),
                        "rhi_mlp_loss_grad")
        return loss.value, g

    def mlp_train(self, X, Y, epochs=1, batch=4096, lr=1e-3):
        """Adam over device tensors X (n x 13), Y (n x 6); returns the last epoch's mean loss."""
        n = X.shape[0]
        (pX, d0), (pY, d1) = _fptr(X, n * RHI_MLP_IN), _fptr(Y, n * RHI_MLP_OUT)
        if not (d0 and d1):
            raise TypeError("training data must be on the device")
        loss = C.c_double()
        self._check(lib().rhi_mlp_train(self.h, pX, pY, n, epochs, batch, lr, C.byref(loss)),
                    "rhi_mlp_train")
        return loss.value

    def set_profiling(self, on, names=None):
        """Per-launch CUDA events on (optionally only for the given kernel names) or off."""
        self._check(lib().rhi_set_profiling_names(self.h, ",".join(names).encode() if names else None),
                    "rhi_set_profiling_names")
        return self._check(lib().rhi_set_profiling(self.h, int(on)), "rhi_set_profiling")

    def kernel_times(self):
        n = lib().rhi_kernel_times(self.h, 0, None, None, None)
        if n <= 0:
            return {}
        names = C.create_string_buffer(48 * n)
        ms = (C.c_double * n)()
        cnt = (C.c_int * n)()
        lib().rhi_kernel_times(self.h, n, names, ms, cnt)
        raw = names.raw
        return {raw[48 * i:48 * i + 48].split(b"\0")[0].decode(): (ms[i], cnt[i]) for i in range(n)}


def params_for_workload(w, **overrides):
    """rhi_params for a synthetic workload (inputs.Workload): species, scalings, theta and the
    grey constants the library computes for the workload's spectrum."""
    p = rhi_params_default(w.ns)
    p.y_he = w.y_he
    if w.model == "lte":
        p.model = RHI_MODEL_LTE
        p.kappa_total, p.kappa_planck, p.mu = w.kappa_total, w.kappa_planck, w.mu
    p.theta = w.theta
    p.u_e, p.u_n, p.u_E = w.u_e, w.u_n, w.u_E
    kind, par = w.spectrum
    spec = {"mono": RHI_SPECTRUM_MONO, "blackbody": RHI_SPECTRUM_BLACKBODY,
            "powerlaw": RHI_SPECTRUM_POWERLAW}[kind]
    g = rhi_grey_constants(spec, par, w.ns)
    for X in range(3):
        p.sk[X], p.pgam[X], p.ph[X] = g["sk"][X], g["pgam"][X], g["ph"][X]
    p.photon_energy = g["eps"]
    for k, v in overrides.items():
        if k in ("sk", "pgam", "ph"):
            for X in range(3):
                getattr(p, k)[X] = v[X]
        else:
            setattr(p, k, v)
    return p


def solver_for_workload(w, stream=None, sources=True, **overrides):
    """A Solver holding the workload's initial state and point sources (host marshalling)."""
    p = params_for_workload(w, **overrides)
    kinds = {"zero_flux": RHI_BC_ZERO_FLUX, "periodic": RHI_BC_PERIODIC,
             "dirichlet": RHI_BC_DIRICHLET}
    bc = [kinds[b] for b in w.bc]
    s = Solver(w.nx, w.ny, w.nz, w.dx, p, bc=bc, stream=stream, bc_value=w.bc_value)
    st = w.state()
    s.set_state(st["E"], st["e"], np.ascontiguousarray(st["n"]).ravel() if w.ns else None,
                np.ascontiguousarray(w.nH.ravel()))
    if sources and len(w.src_rate):
        s.set_sources(w.src_ijk, w.src_rate)
    return s
