"""ctypes binding of librsc.so (the C ABI declared in include/rsc.h).

Argument marshalling only: every stage of the step, the Jacobian action and
Newton-GMRES runs in the library's CUDA kernels.  Device buffers are torch
tensors (float64, contiguous, on the context's device); the CUDA stream is
torch's current stream when the context is created.  There is no CPU
fallback: a missing library raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librsc.so")

RSC_FP64, RSC_MIXED = 0, 1
STATUS = {0: "RSC_OK", 1: "RSC_EINVAL", 2: "RSC_ENOMEM", 3: "RSC_ECUDA", 4: "RSC_ENOCONV",
          5: "RSC_ENAN", 6: "RSC_ESINGULAR", 7: "RSC_ETIMEOUT", 8: "RSC_ERESOLUTION"}
MAX_HISTORY = 64

# Every symbol of include/rsc.h.
EXPORTS = ("rsc_create", "rsc_destroy", "rsc_set_params", "rsc_state_size",
           "rsc_conductive_state", "rsc_step", "rsc_step_host", "rsc_explicit_terms",
           "rsc_apply_jacobian", "rsc_newton_rw", "rsc_newton_rw_host", "rsc_norm2",
           "rsc_last_error", "rsc_status_string", "rsc_abi_version", "rsc_profile_enable",
           "rsc_profile_query", "rsc_kernel_name", "rsc_launch_count", "rsc_norm2_noalloc",
           "rsc_diagnostics", "rsc_step2", "rsc_continuation_predict", "rsc_continue_ra",
           "rsc_batch_create", "rsc_batch_destroy", "rsc_batch_size", "rsc_batch_context",
           "rsc_batch_last_error", "rsc_batch_apply_jacobian", "rsc_batch_newton_rw",
           "rsc_autotune", "rsc_get_tuning", "rsc_set_tuning", "rsc_batch_autotune",
           "rsc_continue_ek", "rsc_spectral_tail", "rsc_regrid", "rsc_refine_params",
           "rsc_implicit_solve", "rsc_factor_block", "rsc_factor_time", "rsc_factor_time_cr")
NORM2_NOALLOC_MAX_N = 8388608
KERNELS = ("radial_eval", "legendre_synth", "fft_products", "legendre_analysis", "rhs_assemble",
           "chain_gemv", "temp_solve", "gmres_dots", "gmres_axpy", "blas1", "chain_sweep",
           "chain_reduced")


class Params(ctypes.Structure):
    _fields_ = [("Ra", ctypes.c_double), ("Ek", ctypes.c_double), ("Pr", ctypes.c_double),
                ("eta", ctypes.c_double), ("L", ctypes.c_int), ("Ms", ctypes.c_int),
                ("Nr", ctypes.c_int), ("precision", ctypes.c_int),
                ("explicit_coriolis", ctypes.c_int)]


class NewtonOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_newton", ctypes.c_int), ("kmax", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("dt_newton", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("products_warps", ctypes.c_int * 2), ("products_lats", ctypes.c_int * 2),
                ("analysis_radii", ctypes.c_int * 2),
                ("analysis_chunk", ctypes.c_int * 2),
                ("synth_radii", ctypes.c_int), ("rhs_pairs", ctypes.c_int * 2),
                ("chain_cluster", ctypes.c_int), ("analysis_tc", ctypes.c_int),
                ("chain_async", ctypes.c_int), ("chain_df", ctypes.c_int),
                ("chain_df_cluster", ctypes.c_int), ("krylov_split", ctypes.c_int),
                ("chain_parts", ctypes.c_int), ("factor_gpu", ctypes.c_int),
                ("refine", ctypes.c_int), ("synth_pipe", ctypes.c_int),
                ("chain_cr", ctypes.c_int), ("ms", ctypes.c_double * 6)]

    def as_dict(self):
        return {"products_warps": list(self.products_warps),
                "products_lats": list(self.products_lats),
                "analysis_radii": list(self.analysis_radii),
                "analysis_chunk": list(self.analysis_chunk), "synth_radii": self.synth_radii,
                "rhs_pairs": list(self.rhs_pairs), "chain_cluster": self.chain_cluster,
                "analysis_tc": self.analysis_tc, "chain_async": self.chain_async,
                "chain_df": self.chain_df, "chain_df_cluster": self.chain_df_cluster,
                "krylov_split": self.krylov_split, "chain_parts": self.chain_parts,
                "factor_gpu": self.factor_gpu, "refine": self.refine,
                "synth_pipe": self.synth_pipe, "chain_cr": self.chain_cr,
                "ms": list(self.ms)}


class ContinuationOpts(ctypes.Structure):
    _fields_ = [("Ra0", ctypes.c_double), ("Ra1", ctypes.c_double), ("Ra_end", ctypes.c_double),
                ("n_opt", ctypes.c_int), ("gamma", ctypes.c_double), ("max_points", ctypes.c_int),
                ("retries", ctypes.c_int), ("newton", NewtonOpts)]


class ContinuationPoint(ctypes.Structure):
    _fields_ = [("Ra", ctypes.c_double), ("C", ctypes.c_double), ("KE", ctypes.c_double),
                ("Nu_in", ctypes.c_double), ("Nu_out", ctypes.c_double),
                ("residual", ctypes.c_double), ("newton_iterations", ctypes.c_int),
                ("gmres_total", ctypes.c_int), ("mode", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class EkContinuationOpts(ctypes.Structure):
    _fields_ = [("Ek0", ctypes.c_double), ("Ek1", ctypes.c_double), ("Ek_end", ctypes.c_double),
                ("ra_coef", ctypes.c_double), ("n_opt", ctypes.c_int), ("gamma", ctypes.c_double),
                ("max_points", ctypes.c_int), ("retries", ctypes.c_int),
                ("tail_threshold", ctypes.c_double), ("newton", NewtonOpts)]


class EkPoint(ctypes.Structure):
    _fields_ = [("Ek", ctypes.c_double), ("Ra", ctypes.c_double), ("C", ctypes.c_double),
                ("KE", ctypes.c_double), ("Nu_in", ctypes.c_double), ("Nu_out", ctypes.c_double),
                ("residual", ctypes.c_double), ("cheb_tail", ctypes.c_double),
                ("sh_tail", ctypes.c_double), ("newton_iterations", ctypes.c_int),
                ("gmres_total", ctypes.c_int), ("mode", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class NewtonReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("gmres_total", ctypes.c_int),
                ("residual", ctypes.c_double), ("C", ctypes.c_double),
                ("residual_history", ctypes.c_double * MAX_HISTORY),
                ("gmres_history", ctypes.c_int * MAX_HISTORY), ("seconds", ctypes.c_double)]

    def as_dict(self):
        it = self.iterations
        return {"iterations": it, "gmres_total": self.gmres_total, "residual": self.residual,
                "C": self.C, "residual_history": list(self.residual_history[: it + 1]),
                "gmres_history": list(self.gmres_history[:it]), "seconds": self.seconds}


class RscError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path=LIB_PATH):
    """Load librsc.so (build it with paper_2508_16635_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librsc.so not found at {path}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    sig = {
        "rsc_create": ([ctypes.POINTER(Params), P, ctypes.POINTER(P)], I),
        "rsc_destroy": ([P], I),
        "rsc_set_params": ([P, ctypes.POINTER(Params)], I),
        "rsc_state_size": ([P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(I)], I),
        "rsc_conductive_state": ([P, P], I),
        "rsc_step": ([P, P, D, D, I], I),
        "rsc_step_host": ([P, P, D, D, I], I),
        "rsc_explicit_terms": ([P, P, P], I),
        "rsc_implicit_solve": ([P, P, P, D], I),
        "rsc_factor_block": ([P, D, I, ctypes.c_long, P], I),
        "rsc_factor_time": ([P, ctypes.POINTER(D), ctypes.POINTER(I)], I),
        "rsc_factor_time_cr": ([P, ctypes.POINTER(D), ctypes.POINTER(I)], I),
        "rsc_apply_jacobian": ([P, P, D, ctypes.c_long, P, P, I, D], I),
        "rsc_newton_rw": ([P, P, ctypes.POINTER(D), ctypes.c_long, ctypes.POINTER(NewtonOpts),
                           ctypes.POINTER(NewtonReport)], I),
        "rsc_newton_rw_host": ([P, P, ctypes.POINTER(D), ctypes.c_long,
                                ctypes.POINTER(NewtonOpts), ctypes.POINTER(NewtonReport)], I),
        "rsc_norm2": ([P, P, ctypes.c_size_t, ctypes.POINTER(D)], I),
        "rsc_last_error": ([P], ctypes.c_char_p),
        "rsc_status_string": ([I], ctypes.c_char_p),
        "rsc_abi_version": ([], I),
        "rsc_profile_enable": ([P, I], I),
        "rsc_profile_query": ([P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_long),
                               ctypes.POINTER(D), ctypes.POINTER(D)], I),
        "rsc_kernel_name": ([I], ctypes.c_char_p),
        "rsc_launch_count": ([P, ctypes.POINTER(ctypes.c_long)], I),
        "rsc_norm2_noalloc": ([P, ctypes.c_size_t, P, P], I),
        "rsc_step2": ([P, P, D, I], I),
        "rsc_continue_ek": ([P, P, ctypes.POINTER(D), ctypes.c_long,
                             ctypes.POINTER(EkContinuationOpts), P, ctypes.POINTER(I)], I),
        "rsc_spectral_tail": ([P, P, ctypes.POINTER(D), ctypes.POINTER(D)], I),
        "rsc_regrid": ([P, P, P, P], I),
        "rsc_refine_params": ([ctypes.POINTER(Params), D, D, D, D, ctypes.POINTER(Params),
                               ctypes.POINTER(I)], I),
        "rsc_autotune": ([P, ctypes.POINTER(Tuning)], I),
        "rsc_get_tuning": ([P, ctypes.POINTER(Tuning)], I),
        "rsc_set_tuning": ([P, ctypes.POINTER(Tuning)], I),
        "rsc_batch_autotune": ([P], I),
        "rsc_batch_create": ([ctypes.POINTER(Params), I, P, ctypes.POINTER(P)], I),
        "rsc_batch_destroy": ([P], I),
        "rsc_batch_size": ([P, ctypes.POINTER(I)], I),
        "rsc_batch_context": ([P, I, ctypes.POINTER(P)], I),
        "rsc_batch_last_error": ([P], ctypes.c_char_p),
        "rsc_batch_apply_jacobian": ([P, P, P, P, P, P, I, D], I),
        "rsc_batch_newton_rw": ([P, P, P, P, ctypes.POINTER(NewtonOpts), P, P], I),
        "rsc_continuation_predict": ([P, P, I, I, I, D, D, ctypes.POINTER(I), ctypes.POINTER(D), P], I),
        "rsc_continue_ra": ([P, P, ctypes.POINTER(D), ctypes.c_long, ctypes.POINTER(ContinuationOpts),
                             P, ctypes.POINTER(I)], I),
        "rsc_diagnostics": ([P, P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class RotatingShell:
    """One problem on the GPU: parameters, truncation, tables and factorisations."""

    def __init__(self, L, Ms, Nr, Ek, Ra, Pr=1.0, eta=0.35, precision="fp64", device=None,
                 coriolis="implicit"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("RotatingShell needs a CUDA device")
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        self.lib = load_library()
        if coriolis not in ("implicit", "explicit"):
            raise ValueError(coriolis)
        self.params = Params(Ra, Ek, Pr, eta, L, Ms, Nr,
                             RSC_MIXED if precision == "mixed" else RSC_FP64,
                             1 if coriolis == "explicit" else 0)
        self.L, self.Ms, self.Nr = L, Ms, Nr
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            st = self.lib.rsc_create(ctypes.byref(self.params), ctypes.c_void_p(stream),
                                     ctypes.byref(self._ctx))
        self._check(st)
        n = ctypes.c_size_t()
        P = ctypes.c_int()
        self._check(self.lib.rsc_state_size(self._ctx, ctypes.byref(n), ctypes.byref(P)))
        self.n, self.P = n.value, P.value

    # ---- helpers -----------------------------------------------------------
    def _check(self, st):
        if st != 0:
            msg = self.lib.rsc_last_error(self._ctx).decode() if self._ctx else ""
            raise RscError(st, msg)

    def _vec(self, t, count=1):
        torch = self.torch
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("expected a contiguous float64 CUDA tensor")
        if t.numel() != self.n * count:
            raise ValueError(f"expected {self.n * count} doubles, got {t.numel()}")
        return _ptr(t)

    def new_state(self):
        return self.torch.zeros(self.n, dtype=self.torch.float64, device=self.device)

    @classmethod
    def _borrow(cls, lib, ctx, params, device):
        """A view of a context owned elsewhere (an instance of a Batch)."""
        import torch
        self = cls.__new__(cls)
        self.torch, self.device, self.lib, self.params = torch, device, lib, params
        self.L, self.Ms, self.Nr = params.L, params.Ms, params.Nr
        self._ctx = ctx
        self._owned = False
        n, P = ctypes.c_size_t(), ctypes.c_int()
        self._check(lib.rsc_state_size(ctx, ctypes.byref(n), ctypes.byref(P)))
        self.n, self.P = n.value, P.value
        return self

    def close(self):
        if self._ctx and getattr(self, "_owned", True):
            self.lib.rsc_destroy(self._ctx)
        self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the C ABI -----------------------------------------------------------
    def set_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        self._check(self.lib.rsc_set_params(self._ctx, ctypes.byref(self.params)))

    def conductive_state(self):
        U = self.new_state()
        self._check(self.lib.rsc_conductive_state(self._ctx, _ptr(U)))
        return U

    def step(self, U, C=0.0, dt=1e-4, nsteps=1):
        self._check(self.lib.rsc_step(self._ctx, self._vec(U), C, dt, nsteps))
        return U

    def step2(self, U, dt=1e-4, nsteps=1):
        """Second-order steps in the laboratory frame (rsc_step2), in place."""
        self._check(self.lib.rsc_step2(self._ctx, self._vec(U), dt, nsteps))
        return U

    def step_host(self, U_host, C=0.0, dt=1e-4, nsteps=1):
        """U_host: contiguous float64 numpy array or pinned CPU tensor (updated in place)."""
        ptr = U_host.ctypes.data if hasattr(U_host, "ctypes") else U_host.data_ptr()
        self._check(self.lib.rsc_step_host(self._ctx, ctypes.c_void_p(ptr), C, dt, nsteps))
        return U_host

    def explicit_terms(self, U):
        N = self.new_state()
        self._check(self.lib.rsc_explicit_terms(self._ctx, self._vec(U), _ptr(N)))
        return N

    def implicit_solve(self, rhs, dt, out=None):
        """x = (M/dt + K)^-1 rhs (rsc_implicit_solve); rhs holds values at the collocation
        radii in the state layout, x Chebyshev coefficients."""
        if out is None:
            out = self.torch.empty_like(rhs)
        self._check(self.lib.rsc_implicit_solve(self._ctx, self._vec(rhs), self._vec(out), dt))
        return out

    def factor_block(self, dt, which, index):
        """One factor block as a numpy array (rsc_factor_block): which in "G", "H", "W"
        (complex Nr x Nr, block `index` over all chains), "T" (real, degree `index`), or the
        odd-even reduced chains' "Dinv" (odd block `index`), "Gr", "Hr", "Wr" (reduced block
        `index`) of a mixed context."""
        import numpy as np
        w = {"G": 0, "H": 1, "W": 2, "T": 3, "Dinv": 4, "Gr": 5, "Hr": 6, "Wr": 7}[which]
        Nr = self.Nr
        buf = np.empty(Nr * Nr * (1 if w == 3 else 2))
        self._check(self.lib.rsc_factor_block(self._ctx, dt, w, index,
                                              ctypes.c_void_p(buf.ctypes.data)))
        if w == 3:
            return buf.reshape(Nr, Nr)
        return (buf[0::2] + 1j * buf[1::2]).reshape(Nr, Nr)

    def factor_time(self):
        """(seconds, on_gpu) of the last factorisation (rsc_factor_time)."""
        sec, on = ctypes.c_double(), ctypes.c_int()
        self._check(self.lib.rsc_factor_time(self._ctx, ctypes.byref(sec), ctypes.byref(on)))
        return sec.value, bool(on.value)

    def factor_time_cr(self):
        """(seconds, on_gpu) of the last factorisation of the odd-even reduced chains
        (rsc_factor_time_cr)."""
        sec, on = ctypes.c_double(), ctypes.c_int()
        self._check(self.lib.rsc_factor_time_cr(self._ctx, ctypes.byref(sec), ctypes.byref(on)))
        return sec.value, bool(on.value)

    def apply_jacobian(self, U, C, J, u, dt, out=None):
        count = u.numel() // self.n
        if out is None:
            out = self.torch.empty_like(u)
        self._check(self.lib.rsc_apply_jacobian(
            self._ctx, self._vec(U), C, -1 if J is None else int(J), self._vec(u, count),
            self._vec(out, count), count, dt))
        return out

    def newton_rw(self, U, C, J, tol=1e-10, max_newton=10, kmax=100, gmres_tol=1e-10,
                  dt_newton=200.0):
        """Newton-GMRES in place on U; returns (C, report dict, status)."""
        opts = NewtonOpts(tol, max_newton, kmax, gmres_tol, dt_newton)
        rep = NewtonReport()
        Cv = ctypes.c_double(C)
        st = self.lib.rsc_newton_rw(self._ctx, self._vec(U), ctypes.byref(Cv),
                                    -1 if J is None else int(J), ctypes.byref(opts),
                                    ctypes.byref(rep))
        if st not in (0, 4):
            self._check(st)
        return Cv.value, rep.as_dict(), st

    def continue_ek(self, U, C, J, Ek0, Ek1, Ek_end, ra_coef=0.0, n_opt=3, gamma=400.0,
                    max_points=8, retries=3, tail_threshold=0.0, tol=1e-10, max_newton=12,
                    kmax=200, gmres_tol=1e-10, dt_newton=200.0):
        """Ek continuation at this resolution (rsc_continue_ek); returns (points, C, status),
        status 8 (RSC_ERESOLUTION) when the last point is under-resolved."""
        opts = EkContinuationOpts(Ek0, Ek1, Ek_end, ra_coef, n_opt, gamma, max_points, retries,
                                  tail_threshold,
                                  NewtonOpts(tol, max_newton, kmax, gmres_tol, dt_newton))
        pts = (EkPoint * max_points)()
        npts = ctypes.c_int(0)
        Cv = ctypes.c_double(C)
        st = self.lib.rsc_continue_ek(self._ctx, self._vec(U), ctypes.byref(Cv),
                                      -1 if J is None else int(J), ctypes.byref(opts),
                                      ctypes.cast(pts, ctypes.c_void_p), ctypes.byref(npts))
        if st not in (0, 4, 8):
            self._check(st)
        return [pts[i].as_dict() for i in range(npts.value)], Cv.value, st

    def spectral_tail(self, U):
        """(Chebyshev, spherical-harmonic) tail ratios of U - U_cond (rsc_spectral_tail)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.rsc_spectral_tail(self._ctx, self._vec(U), ctypes.byref(a),
                                               ctypes.byref(b)))
        return a.value, b.value

    def regrid_from(self, other, U_other):
        """This context's state holding `other`'s state U_other (rsc_regrid)."""
        out = self.new_state()
        self._check(self.lib.rsc_regrid(other._ctx, other._vec(U_other), self._ctx, _ptr(out)))
        return out

    def phase_slot(self, M, k):
        """Index of Im T at (l = m = M, Chebyshev degree k) in this layout."""
        a = M // self.Ms
        p = a * (self.L + 1) - self.Ms * a * (a - 1) // 2
        return ((2 * self.P + p) * self.Nr + k) * 2 + 1

    def autotune(self):
        """Pick the launch shapes by timing (rsc_autotune); returns them as a dict."""
        t = Tuning()
        self._check(self.lib.rsc_autotune(self._ctx, ctypes.byref(t)))
        return t.as_dict()

    def tuning(self):
        t = Tuning()
        self._check(self.lib.rsc_get_tuning(self._ctx, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, d):
        t = Tuning()
        t.products_warps[:] = d["products_warps"]
        t.products_lats[:] = d.get("products_lats", [1, 1])
        t.analysis_radii[:] = d["analysis_radii"]
        t.analysis_chunk[:] = d.get("analysis_chunk", [16, 16])
        t.synth_radii = d["synth_radii"]
        t.rhs_pairs[:] = d["rhs_pairs"]
        t.chain_cluster = d["chain_cluster"]
        t.chain_async = d.get("chain_async", 0)
        t.analysis_tc = d.get("analysis_tc", 0)
        cur = self.tuning()   # fields absent from d keep the context's current values
        t.chain_df = d.get("chain_df", cur["chain_df"])
        t.chain_df_cluster = d.get("chain_df_cluster", cur["chain_df_cluster"])
        t.krylov_split = d.get("krylov_split", cur["krylov_split"])
        t.chain_parts = d.get("chain_parts", cur["chain_parts"])
        t.factor_gpu = d.get("factor_gpu", cur["factor_gpu"])
        t.refine = d.get("refine", cur["refine"])
        t.synth_pipe = d.get("synth_pipe", cur["synth_pipe"])
        t.chain_cr = d.get("chain_cr", cur["chain_cr"])
        self._check(self.lib.rsc_set_tuning(self._ctx, ctypes.byref(t)))

    def continue_ra(self, U, C, J, Ra0, Ra1, Ra_end, n_opt=4, gamma=20.0, max_points=8,
                    retries=3, tol=1e-10, max_newton=12, kmax=200, gmres_tol=1e-10,
                    dt_newton=200.0):
        """Ra continuation (rsc_continue_ra) from the estimate U at Ra0; U returns the last
        wave.  Returns (list of point dicts, last C, status)."""
        opts = ContinuationOpts(Ra0, Ra1, Ra_end, n_opt, gamma, max_points, retries,
                                NewtonOpts(tol, max_newton, kmax, gmres_tol, dt_newton))
        pts = (ContinuationPoint * max_points)()
        npts = ctypes.c_int(0)
        Cv = ctypes.c_double(C)
        st = self.lib.rsc_continue_ra(self._ctx, self._vec(U), ctypes.byref(Cv),
                                      -1 if J is None else int(J), ctypes.byref(opts),
                                      ctypes.cast(pts, ctypes.c_void_p), ctypes.byref(npts))
        if st not in (0, 4):
            self._check(st)
        return [pts[i].as_dict() for i in range(npts.value)], Cv.value, st

    def newton_rw_host(self, U_host, C, J, tol=1e-10, max_newton=10, kmax=100,
                       gmres_tol=1e-10, dt_newton=200.0):
        opts = NewtonOpts(tol, max_newton, kmax, gmres_tol, dt_newton)
        rep = NewtonReport()
        Cv = ctypes.c_double(C)
        ptr = U_host.ctypes.data if hasattr(U_host, "ctypes") else U_host.data_ptr()
        st = self.lib.rsc_newton_rw_host(self._ctx, ctypes.c_void_p(ptr), ctypes.byref(Cv),
                                         -1 if J is None else int(J), ctypes.byref(opts),
                                         ctypes.byref(rep))
        if st not in (0, 4):
            self._check(st)
        return Cv.value, rep.as_dict(), st

    def profile(self, on=True, kernels=None):
        """Start / stop per-kernel CUDA-event timing inside the library (clears counters).

        kernels: names to time (default all); events bracket only those launches.
        """
        mask = 0
        if on:
            mask = (1 << len(KERNELS)) - 1 if kernels is None else sum(1 << KERNELS.index(k) for k in kernels)
        self._check(self.lib.rsc_profile_enable(self._ctx, mask))

    def profile_report(self):
        """{kernel: {ms, launches, bytes, flops}} accumulated since profile(True)."""
        out = {}
        for k, name in enumerate(KERNELS):
            ms, n, b, f = ctypes.c_double(), ctypes.c_long(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.rsc_profile_query(self._ctx, k, ctypes.byref(ms), ctypes.byref(n),
                                                   ctypes.byref(b), ctypes.byref(f)))
            out[name] = {"ms": ms.value, "launches": n.value, "bytes": b.value, "flops": f.value}
        return out

    def launch_count(self):
        c = ctypes.c_long()
        self._check(self.lib.rsc_launch_count(self._ctx, ctypes.byref(c)))
        return c.value

    def diagnostics(self, U):
        """(KE, Nu_in, Nu_out) of the device state U (rsc_diagnostics)."""
        ke, ni, no = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.rsc_diagnostics(self._ctx, _ptr(U), ctypes.byref(ke), ctypes.byref(ni),
                                             ctypes.byref(no)))
        return ke.value, ni.value, no.value

    def norm2(self, v):
        out = ctypes.c_double()
        self._check(self.lib.rsc_norm2(self._ctx, _ptr(v), v.numel(), ctypes.byref(out)))
        return out.value


def continuation_predict(Ra, s, n_its, n_opt, gamma, alpha_scale=1.0, lib=None):
    """rsc_continuation_predict (host only): (mode, Ra_new, [a, b, c])."""
    lib = lib or load_library()
    k = len(Ra)
    ra = (ctypes.c_double * k)(*Ra)
    sv = (ctypes.c_double * k)(*s)
    mode, rn, w = ctypes.c_int(0), ctypes.c_double(0.0), (ctypes.c_double * 3)()
    st = lib.rsc_continuation_predict(ra, sv, k, n_its, n_opt, gamma, alpha_scale,
                                      ctypes.byref(mode), ctypes.byref(rn), w)
    if st != 0:
        raise RscError(st, "rsc_continuation_predict rejected its arguments")
    return mode.value, rn.value, list(w)


class Batch:
    """Instances solved together (rsc_batch_*): continuation points in Ra and waves of
    different azimuthal symmetries.  `instances` is a list of dicts with the keyword
    arguments of RotatingShell (L, Ms, Nr, Ek, Ra and optionally Pr, eta, precision,
    coriolis)."""

    def __init__(self, instances, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Batch needs a CUDA device")
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        self.lib = load_library()
        n = len(instances)
        arr = (Params * n)()
        for i, d in enumerate(instances):
            cor = d.get("coriolis", "implicit")
            arr[i] = Params(d["Ra"], d["Ek"], d.get("Pr", 1.0), d.get("eta", 0.35), d["L"], d["Ms"],
                            d["Nr"], RSC_MIXED if d.get("precision", "fp64") == "mixed" else RSC_FP64,
                            1 if cor == "explicit" else 0)
        self._b = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            st = self.lib.rsc_batch_create(arr, n, ctypes.c_void_p(stream), ctypes.byref(self._b))
        if st != 0:
            raise RscError(st, "rsc_batch_create failed")
        self.shells = []
        for i in range(n):
            c = ctypes.c_void_p()
            self._check(self.lib.rsc_batch_context(self._b, i, ctypes.byref(c)))
            self.shells.append(RotatingShell._borrow(self.lib, c, arr[i], self.device))

    def _check(self, st):
        if st != 0:
            raise RscError(st, self.lib.rsc_batch_last_error(self._b).decode())

    def __len__(self):
        return len(self.shells)

    def synchronize(self):
        self.torch.cuda.synchronize(self.device)

    def implicit_solve(self, rhs, dt, out=None):
        """x = (M/dt + K)^-1 rhs (rsc_implicit_solve); rhs holds values at the collocation
        radii in the state layout, x Chebyshev coefficients."""
        if out is None:
            out = self.torch.empty_like(rhs)
        self._check(self.lib.rsc_implicit_solve(self._ctx, self._vec(rhs), self._vec(out), dt))
        return out

    def factor_block(self, dt, which, index):
        """One factor block as a numpy array (rsc_factor_block): which in "G", "H", "W"
        (complex Nr x Nr, block `index` over all chains), "T" (real, degree `index`), or the
        odd-even reduced chains' "Dinv" (odd block `index`), "Gr", "Hr", "Wr" (reduced block
        `index`) of a mixed context."""
        import numpy as np
        w = {"G": 0, "H": 1, "W": 2, "T": 3, "Dinv": 4, "Gr": 5, "Hr": 6, "Wr": 7}[which]
        Nr = self.Nr
        buf = np.empty(Nr * Nr * (1 if w == 3 else 2))
        self._check(self.lib.rsc_factor_block(self._ctx, dt, w, index,
                                              ctypes.c_void_p(buf.ctypes.data)))
        if w == 3:
            return buf.reshape(Nr, Nr)
        return (buf[0::2] + 1j * buf[1::2]).reshape(Nr, Nr)

    def factor_time(self):
        """(seconds, on_gpu) of the last factorisation (rsc_factor_time)."""
        sec, on = ctypes.c_double(), ctypes.c_int()
        self._check(self.lib.rsc_factor_time(self._ctx, ctypes.byref(sec), ctypes.byref(on)))
        return sec.value, bool(on.value)

    def factor_time_cr(self):
        """(seconds, on_gpu) of the last factorisation of the odd-even reduced chains
        (rsc_factor_time_cr)."""
        sec, on = ctypes.c_double(), ctypes.c_int()
        self._check(self.lib.rsc_factor_time_cr(self._ctx, ctypes.byref(sec), ctypes.byref(on)))
        return sec.value, bool(on.value)

    def apply_jacobian(self, U, C, J, u, dt, out=None):
        """Jacobian actions of every instance in one graph launch: u[i] holds `count`
        directions of instance i back to back; returns the list of outputs."""
        n = len(self.shells)
        count = u[0].numel() // self.shells[0].n
        if out is None:
            out = [self.torch.empty_like(x) for x in u]
        P = ctypes.c_void_p
        pU = (P * n)(*[self.shells[i]._vec(U[i]) for i in range(n)])
        pu = (P * n)(*[self.shells[i]._vec(u[i], count) for i in range(n)])
        po = (P * n)(*[self.shells[i]._vec(out[i], count) for i in range(n)])
        cC = (ctypes.c_double * n)(*C)
        cJ = (ctypes.c_long * n)(*[-1 if j is None else int(j) for j in J])
        c = lambda a: ctypes.cast(a, P)
        self._check(self.lib.rsc_batch_apply_jacobian(self._b, c(pU), c(cC), c(cJ), c(pu), c(po),
                                                      count, dt))
        return out

    def autotune(self):
        """rsc_batch_autotune: tune each distinct shape once; returns the instances' shapes."""
        self._check(self.lib.rsc_batch_autotune(self._b))
        return [sh.tuning() for sh in self.shells]

    def newton_rw(self, U, C, J, tol=1e-10, max_newton=10, kmax=100, gmres_tol=1e-10,
                  dt_newton=200.0):
        """Newton-GMRES on every instance at once; returns (drifts, reports, statuses)."""
        n = len(self.shells)
        P = ctypes.c_void_p
        pU = (P * n)(*[self.shells[i]._vec(U[i]) for i in range(n)])
        cC = (ctypes.c_double * n)(*C)
        cJ = (ctypes.c_long * n)(*[-1 if j is None else int(j) for j in J])
        reps = (NewtonReport * n)()
        sts = (ctypes.c_int * n)()
        opts = NewtonOpts(tol, max_newton, kmax, gmres_tol, dt_newton)
        c = lambda a: ctypes.cast(a, P)
        st = self.lib.rsc_batch_newton_rw(self._b, c(pU), c(cC), c(cJ), ctypes.byref(opts),
                                          c(reps), c(sts))
        if st not in (0, 4):
            self._check(st)
        return list(cC), [reps[i].as_dict() for i in range(n)], list(sts)

    def close(self):
        if self._b:
            for sh in self.shells:
                sh._ctx = ctypes.c_void_p()
            self.lib.rsc_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def refine_params(params, cheb_tail, sh_tail, threshold, growth=1.2, lib=None):
    """rsc_refine_params: (new Params, refined bits: 1 radial, 2 angular)."""
    lib = lib or load_library()
    out = Params()
    refined = ctypes.c_int(0)
    st = lib.rsc_refine_params(ctypes.byref(params), cheb_tail, sh_tail, threshold, growth,
                               ctypes.byref(out), ctypes.byref(refined))
    if st != 0:
        raise RscError(st, "rsc_refine_params rejected its arguments")
    return out, refined.value


def follow_ek(shell, U, C, M, k_phase, Ek0, Ek1, Ek_end, tail_threshold=1e-6, growth=1.2,
              max_refinements=4, **kw):
    """Ek continuation with grid refinement (Sec. 4.4): rsc_continue_ek on the current
    resolution; on an under-resolved point, a context refined by rsc_refine_params receives
    the state by rsc_regrid and the continuation resumes from that point's Ek with the same
    step ratio.  The phase slot is Im T at (l = m = M, Chebyshev degree k_phase).  Returns
    (points with the resolution of each, the final shell, its state, C)."""
    points = []
    for r in range(max_refinements + 1):
        pts, C, st = shell.continue_ek(U, C, shell.phase_slot(M, k_phase), Ek0, Ek1, Ek_end,
                                       tail_threshold=tail_threshold, **kw)
        points += [dict(p, L=shell.L, Nr=shell.Nr) for p in pts]
        if st != 8 or r == max_refinements or not pts:
            return points, shell, U, C
        last = pts[-1]
        newp, bits = refine_params(shell.params, last["cheb_tail"], last["sh_tail"],
                                   tail_threshold, growth, shell.lib)
        if bits == 0:
            return points, shell, U, C
        prec = "mixed" if newp.precision == RSC_MIXED else "fp64"
        fine = RotatingShell(newp.L, newp.Ms, newp.Nr, newp.Ek, newp.Ra, newp.Pr, newp.eta,
                             precision=prec, device=shell.device,
                             coriolis="explicit" if newp.explicit_coriolis else "implicit")
        U = fine.regrid_from(shell, U)
        ratio = (pts[-1]["Ek"] / pts[-2]["Ek"]) if len(pts) > 1 else Ek1 / Ek0
        Ek0, Ek1 = last["Ek"], last["Ek"] * ratio
        shell = fine
    return points, shell, U, C
