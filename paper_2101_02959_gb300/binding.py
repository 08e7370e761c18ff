"""ctypes binding of ``include/bidomain.h`` (argument marshalling only).

Every array argument may be a float64 numpy array (host memory: the library
copies it through its own device buffers) or a contiguous float64 CUDA torch
tensor (device memory, used in place).  All computation happens in the CUDA
library; nothing here has a CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

BD_OK = 0
ERRORS = {-1: "BD_ERR_ARG", -2: "BD_ERR_NOT_SPD", -3: "BD_ERR_KRYLOV_MAXIT", -4: "BD_ERR_KRYLOV_DIVERGED",
          -5: "BD_ERR_NEWTON", -6: "BD_ERR_NAN", -7: "BD_ERR_TIMEOUT", -8: "BD_ERR_CUDA", -9: "BD_ERR_NOMEM",
          -10: "BD_ERR_STATE", -11: "BD_ERR_SCRATCH"}
BDDC, FETIDP = 0, 1
PCG, GMRES = 0, 1
PRIMAL = {"V": 0, "VE": 1, "VEF": 2}
SCALING = {"deluxe": 0, "rho": 1}
GEOM_BOX, GEOM_ELLIPSOID = 0, 1
FP64, MIXED = 0, 1

IDX = dict(ELEM_SUB=0, NODE_MULT=1, IFACE_NODES=2, CLS_TYPE=3, CLS_PTR=4, CLS_NODES=5, CLS_SUB_PTR=6,
           CLS_SUBS=7, CLS_DUAL_START=8, SUB_NODE_PTR=9, SUB_NODES=10, SUB_NINT=11, SUB_DUAL_PTR=12,
           SUB_DUAL=13, SUB_PRIMAL_PTR=14, SUB_PRIMAL=15, GAUGE=16)

EXPORTED = ["bd_plan_create", "bd_plan_sizes", "bd_plan_index_sets", "bd_plan_destroy", "bd_options_default",
            "bidomain_setup", "bidomain_sizes", "bidomain_index_sets", "bidomain_set_state",
            "bidomain_get_state", "bidomain_step", "bidomain_gating", "bidomain_residual", "bidomain_linearize",
            "schur_apply", "bddc_apply", "fetidp_apply", "fetidp_operator", "krylov_solve", "bidomain_profile",
            "bidomain_profile_read", "bidomain_launch_count", "schur_apply_noalloc", "bidomain_mlp_sizes",
            "bidomain_mlp_params", "bidomain_mlp_loss_grad", "bidomain_mlp_adam_step",
            "bidomain_mlp_reset", "bidomain_coarse_size", "bidomain_coarse_matrix",
            "bidomain_coarse_solve", "bidomain_autotune", "bidomain_destroy",
            "bidomain_strerror", "bidomain_last_error"]
PROF = dict(rankk=0, panel=1, gemv=2, resid=3)                    # kernel classes
REGIONS = dict(linearize=4, krylov=5, trsv=6, mlp=7, step=8)      # regions of a step


class BdMesh(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("l", C.c_double * 3), ("s", C.c_int * 3), ("elem_mask", C.c_void_p),
                ("geometry", C.c_int), ("axes", C.c_double * 6), ("phi", C.c_double * 2),
                ("theta", C.c_double * 2)]


class BdConductivity(C.Structure):
    _fields_ = [("sigma_i", C.c_double * 3), ("sigma_e", C.c_double * 3)]


class BdIonic(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("G", "eta1", "eta2", "vth", "vp", "chi_cm")]


class BdStimulus(C.Structure):
    _fields_ = [("amp", C.c_double), ("t_on", C.c_double), ("t_off", C.c_double), ("box", C.c_double * 6)]


class BdOptions(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("method", "krylov", "primal", "precision", "gmres_restart", "ksp_max_it",
                                       "newton_max_it", "use_graphs")] + \
               [(k, C.c_double) for k in ("ksp_rtol", "ksp_atol", "ksp_dtol", "snes_rtol", "snes_atol",
                                          "snes_stol")] + \
               [(k, C.c_int) for k in ("learned_guess", "mlp_train_steps", "mlp_warmup", "mlp_epochs")] + \
               [("mlp_lr", C.c_double), ("use_tensor_cores", C.c_int), ("lag_jacobian", C.c_int),
                ("scaling", C.c_int), ("precond_every", C.c_int)]


class BdSolveStats(C.Structure):
    _fields_ = [("its", C.c_int), ("reason", C.c_int), ("res0", C.c_double), ("res", C.c_double),
                ("cond", C.c_double)]


class BdStepStats(C.Structure):
    _fields_ = [("newton_its", C.c_int), ("krylov_its", C.c_int), ("reason", C.c_int), ("pad", C.c_int),
                ("res0", C.c_double), ("res_final", C.c_double), ("cond_max", C.c_double),
                ("guess_used", C.c_int), ("pad2", C.c_int), ("res_guess", C.c_double), ("mlp_loss", C.c_double)]


class BdTuneResult(C.Structure):
    _fields_ = [("outer_panel", C.c_int), ("groups", C.c_int), ("tensor_cores", C.c_int), ("candidates", C.c_int),
                ("best_ms", C.c_double), ("default_ms", C.c_double)]


class BdSizes(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("n_node", "n_elem", "n_sub", "n_cls", "n_iface", "n_dual", "n_primal",
                                       "n_lambda", "gauge_node", "gauge_primal")]


_LIB = None


def load(build_if_missing: bool = False):
    """Load libbidomain.so (raises if it is missing and may not be built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is missing: run paper_2101_02959_gb300.build.build() first")
        _build.build()
    lib = C.CDLL(_build.LIB)
    P, I, D, V = C.c_void_p, C.c_int, C.c_double, None
    sig = {
        "bd_plan_create": (I, [C.POINTER(BdMesh), I, C.POINTER(P)]),
        "bd_plan_sizes": (I, [P, C.POINTER(BdSizes)]),
        "bd_plan_index_sets": (I, [P, I, P, C.c_int64, C.POINTER(C.c_int64)]),
        "bd_plan_destroy": (V, [P]),
        "bd_options_default": (I, [C.POINTER(BdOptions)]),
        "bidomain_setup": (I, [C.POINTER(BdMesh), C.POINTER(BdConductivity), C.POINTER(BdIonic), D,
                               C.POINTER(BdOptions), P, C.POINTER(P)]),
        "bidomain_sizes": (I, [P, C.POINTER(BdSizes)]),
        "bidomain_index_sets": (I, [P, I, P, C.c_int64, C.POINTER(C.c_int64)]),
        "bidomain_set_state": (I, [P, P, P, P, D, I]),
        "bidomain_get_state": (I, [P, P, P, P, C.POINTER(D), I]),
        "bidomain_step": (I, [P, C.POINTER(BdStimulus), C.POINTER(BdStepStats)]),
        "bidomain_gating": (I, [P, P, P, P, P, I]),
        "bidomain_residual": (I, [P, C.POINTER(BdStimulus), D, P, P, P, P, P, P, I]),
        "bidomain_linearize": (I, [P, P, P, P, I]),
        "schur_apply": (I, [P, P, P, I]),
        "bddc_apply": (I, [P, P, P, I]),
        "fetidp_apply": (I, [P, P, P, I]),
        "fetidp_operator": (I, [P, P, P, I]),
        "krylov_solve": (I, [P, P, P, I, C.POINTER(BdSolveStats)]),
        "bidomain_profile": (I, [P, I]),
        "bidomain_profile_read": (I, [P, I, C.POINTER(C.c_double)]),
        "bidomain_launch_count": (C.c_int64, []),
        "schur_apply_noalloc": (I, [P, P, P]),
        "bidomain_mlp_sizes": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
        "bidomain_mlp_params": (I, [P, P, I]),
        "bidomain_mlp_loss_grad": (I, [P, P, P, P, C.POINTER(D), P]),
        "bidomain_mlp_adam_step": (I, [P, P, D]),
        "bidomain_mlp_reset": (I, [P]),
        "bidomain_coarse_size": (I, [P, C.POINTER(I), C.POINTER(I)]),
        "bidomain_coarse_matrix": (I, [P, P, P, P]),
        "bidomain_coarse_solve": (I, [P, P, P, I]),
        "bidomain_autotune": (I, [P, C.POINTER(BdTuneResult)]),
        "bidomain_destroy": (I, [P]),
        "bidomain_strerror": (C.c_char_p, [I]),
        "bidomain_last_error": (C.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def launch_count():
    return int(load().bidomain_launch_count())


class BidomainError(RuntimeError):
    """A non-zero status of the C-ABI; ``stats`` holds the call's statistics when it
    returns any (bidomain_step reports the failed step's Newton and Krylov counts)."""

    def __init__(self, code, where, handle=None, stats=None):
        self.code = code
        self.stats = stats
        try:
            lib = load()
            msg = lib.bidomain_strerror(code).decode()
            detail = lib.bidomain_last_error(handle).decode()
        except (OSError, RuntimeError):  # library not built: the code alone
            msg, detail = "", ""
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})" + (f": {detail}" if detail else ""))


def _check(code, where, handle=None):
    if code != BD_OK:
        raise BidomainError(code, where, handle)


def _mesh(w):
    """bd_mesh of a workload dict; its "mask" (uint8 per element, kept alive by w) is
    passed as elem_mask."""
    mask = w.get("mask")
    m = BdMesh()
    m.n[:] = list(w["n"])
    m.s[:] = list(w["s"])
    ell = w.get("ellipsoid")
    if ell is None:
        m.l[:] = list(w["l"])
    else:
        m.geometry = GEOM_ELLIPSOID
        m.axes[:] = list(ell["axes"])
        m.phi[:] = list(ell["phi"])
        m.theta[:] = list(ell["theta"])
    if mask is not None:
        assert mask.dtype == np.uint8 and mask.flags["C_CONTIGUOUS"] and mask.size == int(np.prod(w["n"]))
    m.elem_mask = None if mask is None else mask.ctypes.data
    return m


def _stim(st):
    s = BdStimulus()
    if st is None:
        return None
    s.amp, s.t_on, s.t_off = st["amp"], st["t_on"], st["t_off"]
    s.box[:] = list(st["box"])
    return s


def _ptr(a, n=None):
    """(pointer, on_device) of a float64 numpy array or CUDA torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "float64 contiguous arrays only"
        if n is not None:
            assert a.size >= n, "array too short"
        return a.ctypes.data, 0
    import torch
    assert isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
    if n is not None:
        assert a.numel() >= n, "tensor too short"
    return a.data_ptr(), 1


def _same_kind(ref, n):
    if isinstance(ref, np.ndarray):
        return np.zeros(n)
    import torch
    return torch.zeros(n, dtype=torch.float64, device=ref.device)


class Plan:
    """Host-only index sets of a mesh and partition (no GPU needed)."""

    def __init__(self, w, primal=None):
        lib = load()
        self._lib = lib
        self._h = C.c_void_p()
        _check(lib.bd_plan_create(C.byref(_mesh(w)), PRIMAL[primal or w["primal"]], C.byref(self._h)),
               "bd_plan_create")

    def sizes(self):
        s = BdSizes()
        _check(self._lib.bd_plan_sizes(self._h, C.byref(s)), "bd_plan_sizes")
        return {k: getattr(s, k) for k, _ in BdSizes._fields_}

    def index_set(self, name):
        return _index_set(self._lib.bd_plan_index_sets, self._h, name)

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.bd_plan_destroy(self._h)
            self._h = None


def _index_set(fn, h, name):
    n = C.c_int64()
    _check(fn(h, IDX[name], None, 0, C.byref(n)), "index_sets")
    out = np.zeros(max(n.value, 1), np.int64)
    _check(fn(h, IDX[name], out.ctypes.data, out.size, C.byref(n)), "index_sets")
    return out[:n.value]


def options(method="bddc", krylov="pcg", primal="VE", precision="fp64", **kw):
    lib = load()
    o = BdOptions()
    lib.bd_options_default(C.byref(o))
    o.method = {"bddc": BDDC, "fetidp": FETIDP}[method]
    o.krylov = {"pcg": PCG, "gmres": GMRES}[krylov]
    o.primal = PRIMAL[primal]
    o.precision = {"fp64": FP64, "mixed": MIXED}[precision]
    for k, v in kw.items():
        setattr(o, k, SCALING[v] if k == "scaling" and isinstance(v, str) else v)
    return o


class Solver:
    """One solver handle (bidomain_setup ... bidomain_destroy)."""

    def __init__(self, w, sigma_i, sigma_e, ionic, tau, stream=None, **opt):
        lib = load()
        self._lib = lib
        self.w = w
        opt.setdefault("primal", w.get("primal", "VE"))
        self.opts = options(**opt)
        cond = BdConductivity()
        cond.sigma_i[:] = list(sigma_i)
        cond.sigma_e[:] = list(sigma_e)
        ion = BdIonic(*[ionic[k] for k in ("G", "eta1", "eta2", "vth", "vp", "chi_cm")])
        self._h = C.c_void_p()
        st = None if stream is None else C.c_void_p(stream)
        self._check(lib.bidomain_setup(C.byref(_mesh(w)), C.byref(cond), C.byref(ion), float(tau), C.byref(self.opts),
                                  st, C.byref(self._h)), "bidomain_setup")
        s = BdSizes()
        self._check(lib.bidomain_sizes(self._h, C.byref(s)), "bidomain_sizes")
        self.sizes = {k: getattr(s, k) for k, _ in BdSizes._fields_}
        self.N = self.sizes["n_node"]

    def _check(self, code, where):
        _check(code, where, getattr(self, "_h", None))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bidomain_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def index_set(self, name):
        return _index_set(self._lib.bidomain_index_sets, self._h, name)

    def set_state(self, ui, ue, w, t=0.0):
        (a, d), (b, _), (c, _) = _ptr(ui, self.N), _ptr(ue, self.N), _ptr(w, self.N)
        self._check(self._lib.bidomain_set_state(self._h, a, b, c, float(t), d), "bidomain_set_state")

    def get_state(self, like=None):
        like = np.zeros(1) if like is None else like
        ui, ue, w = (_same_kind(like, self.N) for _ in range(3))
        t = C.c_double()
        d = _ptr(ui)[1]
        self._check(self._lib.bidomain_get_state(self._h, _ptr(ui)[0], _ptr(ue)[0], _ptr(w)[0], C.byref(t), d),
               "bidomain_get_state")
        return ui, ue, w, t.value

    def get_state_into(self, ui, ue, w):
        """Download the state into caller-owned arrays (host numpy or CUDA tensors); returns t."""
        t = C.c_double()
        (a, d), (b, _), (c, _) = _ptr(ui, self.N), _ptr(ue, self.N), _ptr(w, self.N)
        self._check(self._lib.bidomain_get_state(self._h, a, b, c, C.byref(t), d), "bidomain_get_state")
        return t.value

    def step(self, stim=None):
        st = BdStepStats()
        s = _stim(stim)
        code = self._lib.bidomain_step(self._h, None if s is None else C.byref(s), C.byref(st))
        out = {k: getattr(st, k) for k, _ in BdStepStats._fields_ if not k.startswith("pad")}
        if code != BD_OK:
            raise BidomainError(code, "bidomain_step", self._h, stats=out)
        return out

    def gating(self, ui, ue, w):
        out = _same_kind(ui, self.N)
        (a, d), (b, _), (c, _), (o, _) = _ptr(ui, self.N), _ptr(ue, self.N), _ptr(w, self.N), _ptr(out, self.N)
        self._check(self._lib.bidomain_gating(self._h, a, b, c, o, d), "bidomain_gating")
        return out

    def residual(self, stim, t_next, ui, ue, w_next, ui_n, ue_n):
        out = _same_kind(ui, 2 * self.N)
        ps = [_ptr(x, self.N) for x in (ui, ue, w_next, ui_n, ue_n)]
        s = _stim(stim)
        self._check(self._lib.bidomain_residual(self._h, None if s is None else C.byref(s), float(t_next),
                                           *[p for p, _ in ps], _ptr(out)[0], ps[0][1]), "bidomain_residual")
        return out

    def linearize(self, ui, ue, w_next):
        (a, d), (b, _), (c, _) = _ptr(ui, self.N), _ptr(ue, self.N), _ptr(w_next, self.N)
        self._check(self._lib.bidomain_linearize(self._h, a, b, c, d), "bidomain_linearize")

    def _apply(self, fn, x, n, name):
        out = _same_kind(x, n)
        p, d = _ptr(x, n)
        self._check(fn(self._h, p, _ptr(out)[0], d), name)
        return out

    def schur_apply(self, x):
        return self._apply(self._lib.schur_apply, x, self.sizes["n_iface"], "schur_apply")

    def bddc_apply(self, r):
        return self._apply(self._lib.bddc_apply, r, self.sizes["n_iface"], "bddc_apply")

    def fetidp_apply(self, lam):
        return self._apply(self._lib.fetidp_apply, lam, self.sizes["n_lambda"], "fetidp_apply")

    def fetidp_operator(self, lam):
        return self._apply(self._lib.fetidp_operator, lam, self.sizes["n_lambda"], "fetidp_operator")

    def profile(self, enable=True):
        """True / 1: kernel classes and regions; 2: regions only; False / 0: off."""
        mode = 2 if enable == 2 else (1 if enable else 0)
        self._check(self._lib.bidomain_profile(self._h, mode), "bidomain_profile")

    def profile_read(self, which):
        out = (C.c_double * 4)()
        idx = PROF[which] if which in PROF else REGIONS[which]
        self._check(self._lib.bidomain_profile_read(self._h, idx, out), "bidomain_profile_read")
        return dict(launches=int(out[0]), ms=out[1], flops=out[2], bytes=out[3])

    def autotune(self):
        r = BdTuneResult()
        self._check(self._lib.bidomain_autotune(self._h, C.byref(r)), "bidomain_autotune")
        return {k: getattr(r, k) for k, _ in BdTuneResult._fields_}

    def mlp_sizes(self):
        v = [C.c_int() for _ in range(4)]
        self._check(self._lib.bidomain_mlp_sizes(self._h, *[C.byref(x) for x in v]), "bidomain_mlp_sizes")
        return dict(zip(("n_in", "n_hidden", "n_out", "batch"), (x.value for x in v)))

    def mlp_params(self, w=None):
        """Packed float32 parameters: upload `w` when given, else download."""
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float32)
            self._check(self._lib.bidomain_mlp_params(self._h, w.ctypes.data, 1), "bidomain_mlp_params")
            return w
        sz = self.mlp_sizes()
        n = sz["n_hidden"] * (sz["n_in"] + 1) + sz["n_hidden"] * (sz["n_hidden"] + 1) + \
            sz["n_out"] * (sz["n_hidden"] + 1)
        out = np.zeros(n, np.float32)
        self._check(self._lib.bidomain_mlp_params(self._h, out.ctypes.data, 0), "bidomain_mlp_params")
        return out

    def mlp_loss_grad(self, X, T, mask):
        X, T, mask = (np.ascontiguousarray(a, dtype=np.float32) for a in (X, T, mask))
        w = self.mlp_params()
        g = np.zeros_like(w)
        loss = C.c_double()
        self._check(self._lib.bidomain_mlp_loss_grad(self._h, X.ctypes.data, T.ctypes.data, mask.ctypes.data,
                                                C.byref(loss), g.ctypes.data), "bidomain_mlp_loss_grad")
        return loss.value, g

    def mlp_adam_step(self, grad, lr):
        """One Adam step of the packed parameters with the packed gradient ``grad``."""
        g = np.ascontiguousarray(grad, dtype=np.float32)
        self._check(self._lib.bidomain_mlp_adam_step(self._h, g.ctypes.data, float(lr)), "bidomain_mlp_adam_step")

    def mlp_reset(self):
        """Back to the untrained network (initial weights, zero Adam state, no history)."""
        self._check(self._lib.bidomain_mlp_reset(self._h), "bidomain_mlp_reset")

    def coarse_matrix(self):
        """S_PiPi of the current Jacobian as (rowptr, col, val) numpy arrays (FP64 CSR)."""
        np_, nnz = C.c_int(), C.c_int()
        self._check(self._lib.bidomain_coarse_size(self._h, C.byref(np_), C.byref(nnz)), "bidomain_coarse_size")
        ptr = np.zeros(np_.value + 1, np.int32)
        col = np.zeros(max(nnz.value, 1), np.int32)
        val = np.zeros(max(nnz.value, 1))
        self._check(self._lib.bidomain_coarse_matrix(self._h, ptr.ctypes.data, col.ctypes.data, val.ctypes.data),
                    "bidomain_coarse_matrix")
        return ptr, col[:nnz.value], val[:nnz.value]

    def coarse_solve(self, c, nref=-1):
        """The coarse solve z = S_PiPi^-1 c as the preconditioner performs it."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        z = np.zeros_like(c)
        self._check(self._lib.bidomain_coarse_solve(self._h, c.ctypes.data, z.ctypes.data, int(nref)),
                    "bidomain_coarse_solve")
        return z

    def krylov_solve(self, f):
        out = _same_kind(f, 2 * self.N)
        st = BdSolveStats()
        p, d = _ptr(f, 2 * self.N)
        code = self._lib.krylov_solve(self._h, p, _ptr(out)[0], d, C.byref(st))
        stats = {k: getattr(st, k) for k, _ in BdSolveStats._fields_}
        self._check(code, "krylov_solve")
        return out, stats
