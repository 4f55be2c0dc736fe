"""Thin ctypes binding of libefe (include/efe.h): argument marshalling only.

Every computation runs in the CUDA library; this module only converts Python
and torch arguments into the C structs and raw pointers the ABI expects.  It
raises if the compiled library is missing -- there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libefe.so")

EFE_FP64, EFE_FP32, EFE_BF16 = 0, 1, 2
EFE_FILTER_RESIDUAL, EFE_FILTER_STANDARD, EFE_FILTER_KEEP_PRECISION = 0, 1, 2
PRECISIONS = {"fp64": EFE_FP64, "fp32": EFE_FP32, "bf16": EFE_BF16}
STATUS = {0: "EFE_OK", 1: "EFE_ERR_ARG", 2: "EFE_ERR_CUDA", 3: "EFE_ERR_NOT_SPD",
          4: "EFE_ERR_NO_CONVERGE", 5: "EFE_ERR_TIMEOUT", 6: "EFE_ERR_OOM", 7: "EFE_ERR_STATE"}


class efe_mesh(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("ncell", ctypes.c_int * 3), ("degree", ctypes.c_int),
                ("nquad", ctypes.c_int)]


class efe_atoms(ctypes.Structure):
    _fields_ = [("natoms", ctypes.c_int), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("zval", ctypes.POINTER(ctypes.c_double))]


class efe_enrichment(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("alpha", ctypes.c_double), ("r_end", ctypes.c_double),
                ("t", ctypes.c_double)]


class efe_psp(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("rc", ctypes.c_double), ("r_trunc", ctypes.c_double),
                ("h", ctypes.POINTER(ctypes.c_double)), ("rloc", ctypes.c_double)]


class efe_dims(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_longlong), ("n_fe_dof", ctypes.c_longlong),
                ("n_rows", ctypes.c_longlong), ("n_quad", ctypes.c_longlong), ("n_enr", ctypes.c_int),
                ("n_proj", ctypes.c_int), ("n_cells", ctypes.c_int), ("ne", ctypes.c_int),
                ("nq", ctypes.c_int), ("grid", ctypes.c_int * 3), ("n_support_nodes", ctypes.c_longlong)]


class efe_stats(ctypes.Structure):
    _fields_ = [("ms_filter", ctypes.c_double), ("ms_rr", ctypes.c_double), ("ms_lanczos", ctypes.c_double),
                ("ms_cell", ctypes.c_double), ("launches", ctypes.c_longlong),
                ("cell_launches", ctypes.c_longlong), ("passes", ctypes.c_int), ("ms_rec", ctypes.c_double),
                ("rec_launches", ctypes.c_longlong)]


SCF_LOG = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                           ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double)


class efe_scf_opts(ctypes.Structure):
    _fields_ = [("cheb_degree", ctypes.c_int), ("temperature", ctypes.c_double), ("mix_beta", ctypes.c_double),
                ("mix_history", ctypes.c_int), ("tol_rho", ctypes.c_double), ("tol_e", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("first_tol", ctypes.c_double), ("first_max_pass", ctypes.c_int),
                ("renormalize", ctypes.c_int), ("kappa", ctypes.c_double), ("poisson_tol", ctypes.c_double),
                ("precision", ctypes.c_int), ("log", SCF_LOG), ("log_user", ctypes.c_void_p),
                ("bf16_resid", ctypes.c_double), ("profile", ctypes.c_int), ("passes", ctypes.c_int),
                ("precond_k2", ctypes.c_double)]


class efe_scf_result(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("F", ctypes.c_double), ("mu", ctypes.c_double), ("drho", ctypes.c_double),
                ("dE", ctypes.c_double), ("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("poisson_iters", ctypes.c_longlong), ("eig", ctypes.POINTER(ctypes.c_double)),
                ("rho_q", ctypes.c_void_p), ("ms_phase", ctypes.c_double * 5)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int
SIGNATURES = {
    "efe_setup": [ctypes.POINTER(efe_mesh), ctypes.POINTER(efe_atoms), ctypes.POINTER(efe_enrichment),
                  ctypes.POINTER(efe_psp), _P, ctypes.POINTER(_P)],
    "efe_destroy": [_P],
    "efe_last_error": [_P],
    "efe_get_dims": [_P, ctypes.POINTER(efe_dims)],
    "efe_get_stats": [_P, ctypes.POINTER(efe_stats)],
    "efe_set_potential": [_P, _P],
    "efe_apply_h": [_P, _P, _P, _I, _I],
    "efe_apply_m": [_P, _P, _P, _I],
    "efe_apply_minv": [_P, _P, _P, _I],
    "efe_lanczos": [_P, _P, _I, _D],
    "efe_filter": [_P, _P, _P, _P, _I, _I, _D, _I, _P],
    "efe_set_cell_storage": [_P, _I],
    "efe_set_poisson_precision": [_P, _I],
    "efe_rayleigh_ritz": [_P, _P, _P, _I, _D, _D],
    "efe_chfsi": [_P, _P, _P, _I, _I, _D, _P, _I, ctypes.c_double, _I, _I, _D, _D, ctypes.POINTER(_I)],
    "efe_filter_host": [_P, _D, _D, _D, _I, _I, _D, _I, _D],
    "efe_filter_standard": [_P, _P, _P, _I, _I, _D, _I, _P],
    "efe_chfsi_kind": [_P, _P, _P, _I, _I, _D, _P, _I, ctypes.c_double, _I, _I, _I, _D, _D,
                       ctypes.POINTER(_I), _D],
    "efe_smeared_charge": [_P, _P],
    "efe_atomic_density": [_P, ctypes.c_double, _P],
    "efe_density": [_P, _P, _I, _D, _P],
    "efe_xc": [_P, _P, _P, _P],
    "efe_poisson": [_P, _P, _P, _P, ctypes.c_double, _I, ctypes.POINTER(_I), _D],
    "efe_fermi": [_P, _D, _I, ctypes.c_double, ctypes.c_double, _D, _D],
    "efe_integrate": [_P, _P, _P, _D],
    "efe_integrate_noalloc": [_P, _P, _P, _D],
    "efe_scf": [_P, ctypes.POINTER(efe_scf_opts), _P, _I, _P, _P, ctypes.POINTER(efe_scf_result)],
    "efe_mlp_create": [_P, _I, ctypes.POINTER(_P)],
    "efe_mlp_destroy": [_P],
    "efe_mlp_last_error": [_P],
    "efe_descriptors": [_P, _P, _P, _I, _P],
    "efe_mlp_forward": [_P, _P, _P, _I, _P],
    "efe_mlp_normalise": [_P, _P, _P, _P, _I],
    "efe_mlp_loss_grad": [_P, _P, _P, _P, _I, _P, _D],
    "efe_mlp_adam": [_P, _P, _P, _P, _P, _I, _P],
    "efe_mlp_train": [_P, _P, _P, _P, _P, _P, _I, _I, _I, _P, _P],
    "efe_mlp_save": [_P, _P, ctypes.c_char_p],
    "efe_mlp_load": [_P, ctypes.c_char_p, _P],
    "efe_density_correction": [_P, _P, _P],
    "efe_fit_correction": [_P, _P, _P, ctypes.c_double, _P],
    "efe_corrected_density": [_P, _P, ctypes.c_double, _P, ctypes.POINTER(_I)],
    "efe_warm_start": [_P, _P, _P, ctypes.c_double, _P, ctypes.POINTER(_I)],
}

MLP_N_DESC, MLP_N_OUT, MLP_N_TRAIN, MLP_N_PARAMS = 32, 8, 38280, 38360


class efe_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]

_lib = None


def load():
    """Load libefe.so (built in-tree by paper_2607_06848_gb300.build).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libefe.so is not built: run `python -m paper_2607_06848_gb300.build` "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = (ctypes.c_char_p if name in ("efe_last_error", "efe_mlp_last_error") else
                      None if name in ("efe_destroy", "efe_mlp_destroy") else ctypes.c_int)
    _lib = lib
    return lib


class EFEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def _ptr(t):
    """Raw device pointer of a contiguous CUDA tensor."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _darr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


class EFE:
    """One EFE discretisation on the current CUDA device (wraps an efe_ctx)."""

    def __init__(self, h, ncell, degree, atoms, zval, enrich=None, psp=None, nquad=0, stream=None):
        import torch
        self.lib = load()
        self._keep = []
        mesh = efe_mesh(float(h), (ctypes.c_int * 3)(*[int(v) for v in ncell]), int(degree), int(nquad))
        xyz, pxyz = _darr(np.asarray(atoms, float).reshape(-1, 3))
        z, pz = _darr(zval)
        self._keep += [xyz, z]
        at = efe_atoms(len(z), pxyz, pz)
        en = efe_enrichment(0, 0.0, 0.0, 0.0)
        if enrich is not None:
            en = efe_enrichment(1, float(enrich["alpha"]), float(enrich["r_end"]), float(enrich["t"]))
        ps = efe_psp(0, 0.0, 0.0, None, 0.8)
        if psp is not None:
            hh, ph = _darr(np.asarray(psp["h"], float).reshape(-1, 2))
            self._keep.append(hh)
            ps = efe_psp(1, float(psp["rc"]), float(psp["r_trunc"]), ph, float(psp.get("rloc", 0.8)))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        ctx = ctypes.c_void_p()
        st = self.lib.efe_setup(ctypes.byref(mesh), ctypes.byref(at), ctypes.byref(en), ctypes.byref(ps),
                                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(ctx))
        if st != 0:
            raise EFEError(st, self.lib.efe_last_error(None).decode())
        self.ctx = ctx
        d = efe_dims()
        self._check(self.lib.efe_get_dims(self.ctx, ctypes.byref(d)))
        self.dims = {k: (list(getattr(d, k)) if k == "grid" else getattr(d, k)) for k, _ in efe_dims._fields_}

    def _check(self, st):
        if st != 0:
            raise EFEError(st, self.lib.efe_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.efe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- marshalling wrappers with the ABI names -------------------------
    def stats(self):
        s = efe_stats()
        self._check(self.lib.efe_get_stats(self.ctx, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in efe_stats._fields_}

    def efe_set_potential(self, veff_q):
        self._check(self.lib.efe_set_potential(self.ctx, _ptr(veff_q)))

    def efe_apply_h(self, X, Y, prec=EFE_FP64):
        self._check(self.lib.efe_apply_h(self.ctx, _ptr(X), _ptr(Y), X.shape[1], prec))

    def efe_apply_m(self, X, Y):
        self._check(self.lib.efe_apply_m(self.ctx, _ptr(X), _ptr(Y), X.shape[1]))

    def efe_apply_minv(self, X, Y):
        self._check(self.lib.efe_apply_minv(self.ctx, _ptr(X), _ptr(Y), X.shape[1]))

    def efe_lanczos(self, u0, k=10):
        out = (ctypes.c_double * 3)()
        self._check(self.lib.efe_lanczos(self.ctx, _ptr(u0), int(k), out))
        return tuple(out)

    def efe_set_cell_storage(self, prec):
        self._check(self.lib.efe_set_cell_storage(self.ctx, int(prec)))

    def efe_set_poisson_precision(self, prec):
        self._check(self.lib.efe_set_poisson_precision(self.ctx, int(prec)))

    def efe_filter(self, V, HV, lam, m, bounds, Vout, prec=EFE_FP64):
        b = (ctypes.c_double * 3)(*[float(x) for x in bounds])
        self._check(self.lib.efe_filter(self.ctx, _ptr(V), _ptr(HV), _ptr(lam), V.shape[1], int(m), b,
                                        int(prec), _ptr(Vout)))

    def efe_filter_standard(self, V, HV, m, bounds, Vout, prec=EFE_FP64):
        b = (ctypes.c_double * 3)(*[float(x) for x in bounds])
        self._check(self.lib.efe_filter_standard(self.ctx, _ptr(V), _ptr(HV), V.shape[1], int(m), b,
                                                 int(prec), _ptr(Vout)))

    def efe_rayleigh_ritz(self, X, HX):
        N = X.shape[1]
        eig = (ctypes.c_double * N)()
        res = (ctypes.c_double * N)()
        self._check(self.lib.efe_rayleigh_ritz(self.ctx, _ptr(X), _ptr(HX), N, eig, res))
        return np.array(eig[:]), np.array(res[:])

    def efe_chfsi(self, X, m, bounds=None, u0=None, max_pass=20, tol=1e-8, nconv=0, prec=EFE_FP64, HX=None):
        N = X.shape[1]
        eig = (ctypes.c_double * N)()
        res = (ctypes.c_double * N)()
        passes = ctypes.c_int(0)
        b = None if bounds is None else (ctypes.c_double * 3)(*[float(x) for x in bounds])
        st = self.lib.efe_chfsi(self.ctx, _ptr(X), _ptr(HX), N, int(m), b, _ptr(u0), int(max_pass),
                                float(tol), int(nconv), int(prec), eig, res, ctypes.byref(passes))
        if st not in (0, 4):
            self._check(st)
        return np.array(eig[:]), np.array(res[:]), passes.value, st == 0

    def efe_chfsi_kind(self, X, m, kind=EFE_FILTER_RESIDUAL, bounds=None, u0=None, max_pass=20, tol=1e-8,
                       nconv=0, prec=EFE_FP64, HX=None):
        """efe_chfsi with a choice of filter; also returns the per-pass max residual."""
        N = X.shape[1]
        eig = (ctypes.c_double * N)()
        res = (ctypes.c_double * N)()
        hist = (ctypes.c_double * max(int(max_pass), 1))()
        passes = ctypes.c_int(0)
        b = None if bounds is None else (ctypes.c_double * 3)(*[float(x) for x in bounds])
        st = self.lib.efe_chfsi_kind(self.ctx, _ptr(X), _ptr(HX), N, int(m), b, _ptr(u0), int(max_pass),
                                     float(tol), int(nconv), int(prec), int(kind), eig, res,
                                     ctypes.byref(passes), hist)
        if st not in (0, 4):
            self._check(st)
        return (np.array(eig[:]), np.array(res[:]), passes.value, st == 0,
                np.array(hist[:passes.value]))

    def efe_filter_host(self, V, HV, lam, m, bounds, prec=EFE_FP64, out=None):
        """Host arrays in and out (the library copies on its stream); out: an optional
        caller-owned (e.g. pinned) host array for V_out."""
        V = np.ascontiguousarray(V, dtype=np.float64)
        HV = np.ascontiguousarray(HV, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        if out is None:
            out = np.empty_like(V)
        if out.shape != V.shape or out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous float64 array shaped like V")
        b = (ctypes.c_double * 3)(*[float(x) for x in bounds])
        self._check(self.lib.efe_filter_host(self.ctx, V.ctypes.data_as(_D), HV.ctypes.data_as(_D),
                                             lam.ctypes.data_as(_D), V.shape[1], int(m), b, int(prec),
                                             out.ctypes.data_as(_D)))
        return out

    # --- SCF pieces --------------------------------------------------------
    def efe_smeared_charge(self, b_q):
        self._check(self.lib.efe_smeared_charge(self.ctx, _ptr(b_q)))

    def efe_atomic_density(self, kappa, rho_q):
        self._check(self.lib.efe_atomic_density(self.ctx, float(kappa), _ptr(rho_q)))

    def efe_density(self, X, occ, rho_q):
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        self._check(self.lib.efe_density(self.ctx, _ptr(X), X.shape[1], occ.ctypes.data_as(_D), _ptr(rho_q)))

    def efe_xc(self, rho_q, vxc_q=None, exc_q=None):
        self._check(self.lib.efe_xc(self.ctx, _ptr(rho_q), _ptr(vxc_q), _ptr(exc_q)))

    def efe_poisson(self, f_q, phi_nodes, phi_q=None, tol=1e-12, max_it=100000):
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        self._check(self.lib.efe_poisson(self.ctx, _ptr(f_q), _ptr(phi_nodes), _ptr(phi_q), float(tol),
                                         int(max_it), ctypes.byref(it), ctypes.byref(rr)))
        return it.value, rr.value

    def efe_fermi(self, eig, n_elec, kT):
        eig = np.ascontiguousarray(eig, dtype=np.float64)
        occ = np.empty_like(eig)
        mu = ctypes.c_double(0.0)
        self._check(self.lib.efe_fermi(self.ctx, eig.ctypes.data_as(_D), len(eig), float(n_elec), float(kT),
                                       ctypes.byref(mu), occ.ctypes.data_as(_D)))
        return mu.value, occ

    def efe_integrate(self, a_q, b_q=None):
        out = ctypes.c_double(0.0)
        self._check(self.lib.efe_integrate(self.ctx, _ptr(a_q), _ptr(b_q), ctypes.byref(out)))
        return out.value

    def efe_integrate_noalloc(self, a_q, b_q=None):
        out = ctypes.c_double(0.0)
        self._check(self.lib.efe_integrate_noalloc(self.ctx, _ptr(a_q), _ptr(b_q), ctypes.byref(out)))
        return out.value

    def efe_scf(self, X, u0, rho0_q=None, rho_out=None, log=None, **opts):
        o = efe_scf_opts(int(opts.get("cheb_degree", 20)), float(opts.get("temperature", 500.0)),
                         float(opts.get("mix_beta", 0.5)), int(opts.get("mix_history", 8)),
                         float(opts.get("tol_rho", 1e-8)), float(opts.get("tol_e", 1e-8)),
                         int(opts.get("max_iter", 60)), float(opts.get("first_tol", 1e-2)),
                         int(opts.get("first_max_pass", 20)), int(opts.get("renormalize", 1)),
                         float(opts.get("kappa", 2.4)), float(opts.get("poisson_tol", 1e-12)),
                         int(opts.get("precision", EFE_FP64)), SCF_LOG(0), None,
                         float(opts.get("bf16_resid", 0.0)), int(opts.get("profile", 0)),
                         int(opts.get("passes", 1)), float(opts.get("precond_k2", 0.0)))
        hist = []
        if log is not None:
            def cb(user, it, E, F, mu, dr, dE, r0):
                rec = dict(it=it, E=E, F=F, mu=mu, drho=dr, dE=dE, resid0=r0)
                hist.append(rec)
                log(rec)
            o.log = SCF_LOG(cb)
        N = X.shape[1]
        eig = (ctypes.c_double * N)()
        res = efe_scf_result()
        res.eig = ctypes.cast(eig, ctypes.POINTER(ctypes.c_double))
        res.rho_q = None if rho_out is None else ctypes.c_void_p(rho_out.data_ptr())
        st = self.lib.efe_scf(self.ctx, ctypes.byref(o), _ptr(X), N, _ptr(u0), _ptr(rho0_q), ctypes.byref(res))
        if st not in (0, 4):
            self._check(st)
        return dict(E=res.E, F=res.F, mu=res.mu, drho=res.drho, dE=res.dE, iters=res.iters,
                    converged=bool(res.converged), poisson_iters=res.poisson_iters, eig=np.array(eig[:]),
                    history=hist, ms_phase=list(res.ms_phase))

    # --- learned warm start (ctx part) -----------------------------------
    def efe_density_correction(self, c, drho_q):
        self._check(self.lib.efe_density_correction(self.ctx, _ptr(c), _ptr(drho_q)))

    def efe_fit_correction(self, rho_q, c, base_q=None, ridge=1e-3):
        self._check(self.lib.efe_fit_correction(self.ctx, _ptr(rho_q), _ptr(base_q), float(ridge), _ptr(c)))

    def efe_corrected_density(self, c, rho_q, kappa=2.4):
        """Returns True when rho_q holds the superposition (fallback)."""
        fb = ctypes.c_int(1)
        self._check(self.lib.efe_corrected_density(self.ctx, _ptr(c), float(kappa), _ptr(rho_q), ctypes.byref(fb)))
        return bool(fb.value)

    def efe_warm_start(self, mlp, theta, rho_q, kappa=2.4):
        """Returns True when rho_q holds the superposition (no network or fallback)."""
        fb = ctypes.c_int(1)
        self._check(self.lib.efe_warm_start(self.ctx, None if mlp is None else mlp.h, _ptr(theta),
                                            float(kappa), _ptr(rho_q), ctypes.byref(fb)))
        return bool(fb.value)


class MLP:
    """Training workspace of the warm-start network (efe_mlp_*): marshalling only."""

    def __init__(self, max_samples, stream=None):
        import torch
        self.lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.lib.efe_mlp_create(ctypes.c_void_p(stream.cuda_stream), int(max_samples), ctypes.byref(h))
        if st != 0:
            raise EFEError(st, self.lib.efe_mlp_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != 0:
            raise EFEError(st, self.lib.efe_mlp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.efe_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def efe_descriptors(self, xyz, zval, D):
        self._check(self.lib.efe_descriptors(self.h, _ptr(xyz), _ptr(zval), xyz.shape[0], _ptr(D)))

    def efe_mlp_forward(self, theta, D, C):
        self._check(self.lib.efe_mlp_forward(self.h, _ptr(theta), _ptr(D), D.shape[0], _ptr(C)))

    def efe_mlp_normalise(self, theta, D, T):
        self._check(self.lib.efe_mlp_normalise(self.h, _ptr(theta), _ptr(D), _ptr(T), D.shape[0]))

    def efe_mlp_loss_grad(self, theta, D, T, grad):
        loss = ctypes.c_double(0.0)
        self._check(self.lib.efe_mlp_loss_grad(self.h, _ptr(theta), _ptr(D), _ptr(T), D.shape[0], _ptr(grad),
                                               ctypes.byref(loss)))
        return loss.value

    def efe_mlp_adam(self, theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        hp = efe_adam(lr, beta1, beta2, eps)
        self._check(self.lib.efe_mlp_adam(self.h, _ptr(theta), _ptr(m), _ptr(v), _ptr(grad), int(t),
                                          ctypes.byref(hp)))

    def efe_mlp_save(self, theta, path):
        self._check(self.lib.efe_mlp_save(self.h, _ptr(theta), os.fsencode(path)))

    def efe_mlp_load(self, path, theta):
        self._check(self.lib.efe_mlp_load(self.h, os.fsencode(path), _ptr(theta)))

    def efe_mlp_train(self, theta, m, v, D, T, steps, loss_hist, t0=0, lr=1e-3, beta1=0.9, beta2=0.999,
                      eps=1e-8):
        hp = efe_adam(lr, beta1, beta2, eps)
        self._check(self.lib.efe_mlp_train(self.h, _ptr(theta), _ptr(m), _ptr(v), _ptr(D), _ptr(T), D.shape[0],
                                           int(steps), int(t0), ctypes.byref(hp), _ptr(loss_hist)))
