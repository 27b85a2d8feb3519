"""Python binding of the GB300 CPTR-FGMRES library (C ABI in include/cptr.h).

Argument marshalling only: every step of the solve runs in the CUDA kernels of libcptr.so.  The
functions mirror the C entry points by name; :class:`Solver` bundles them for torch tensors.
There is no CPU fallback: if libcptr.so is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LIB_PATH = _build.LIB

CPTR_OK, CPTR_NOT_CONVERGED = 0, 1
STATUS = {0: "CPTR_OK", 1: "CPTR_NOT_CONVERGED", -1: "CPTR_EINVAL", -2: "CPTR_ENOMEM", -3: "CPTR_ECUDA",
          -4: "CPTR_EBREAKDOWN", -5: "CPTR_ETIMEOUT", -6: "CPTR_ESINGULAR", -7: "CPTR_ESTATE", -8: "CPTR_ECHECK"}
STAGE1 = {"full": 0, "upper": 1, "lower": 2, "bd": 3, "cpr": 4, "none": 5, "uamg": 6}
STAGE2 = {"ilu0": 0, "none": 1}
SCHUR = {"given": 0, "att": 1, "learned": 2, "diag": 3}
SCHUR_NAMES = {v: k for k, v in SCHUR.items()}
MLP_FEATURES, MLP_HIDDEN, MLP_NPARAM = 16, 64, 5313
SMOOTHER = {"l1": 0, "jacobi": 1}
PRECISION = {"fp64": 0, "mixed": 1}
ILU_ORDER = {"natural": 0, "multicolor": 1}
ILU_SWEEP = {"auto": 0, "levels": 1, "chunked": 2, "paired": 3, "tiled": 4}
DECOUPLE = {"none": 0, "qi": 1, "ti": 2}
U_P, U_T, U_SAT = 0, 1, 2


class cptr_options(ctypes.Structure):
    _fields_ = [("stage1", ctypes.c_int32), ("stage2", ctypes.c_int32), ("schur", ctypes.c_int32),
                ("smoother", ctypes.c_int32), ("omega", ctypes.c_double), ("theta", ctypes.c_double),
                ("n_coarse", ctypes.c_int32), ("max_levels", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_it", ctypes.c_int32), ("dense_max", ctypes.c_int32), ("seed", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("check_every", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("ilu_order", ctypes.c_int32), ("autotune", ctypes.c_int32), ("ilu_sweep", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("tile_y", ctypes.c_int32), ("tile_z", ctypes.c_int32),
                ("decouple", ctypes.c_int32), ("ilu_fill", ctypes.c_int32), ("csr_lanes", ctypes.c_int32),
                ("ilu_group", ctypes.c_int32), ("ilu_lanes", ctypes.c_int32)]


class cptr_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("levels_p", ctypes.c_int32), ("levels_T", ctypes.c_int32), ("schur_used", ctypes.c_int32),
                ("est_rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("op_complexity_p", ctypes.c_double), ("op_complexity_T", ctypes.c_double)]


class cptr_instance(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32), ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("row_weights", ctypes.c_void_p), ("st_vals", ctypes.c_void_p)]


class cptr_model(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("nphase", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("phi", ctypes.c_double), ("grav", ctypes.c_double),
                ("kh", ctypes.c_void_p), ("kv", ctypes.c_void_p)] + \
        [(k, ctypes.c_double) for k in ("kT_const", "kT_rock", "kT_w", "kT_o", "kT_g", "cv_w", "cv_o", "cv_g",
                                        "c_rock", "rho_rock", "mu_o_ref", "beta_mu", "T0", "rho_o_ref", "c_o",
                                        "beta_o", "p0", "gas_M", "mu_g", "corey_n")] + \
        [("n_wells", ctypes.c_int32), ("n_heaters", ctypes.c_int32), ("well_cell", ctypes.c_void_p),
         ("well_kind", ctypes.c_void_p), ("well_a", ctypes.c_void_p), ("well_c", ctypes.c_void_p),
         ("heater_cell", ctypes.c_void_p), ("heater_U", ctypes.c_void_p), ("heater_T", ctypes.c_void_p),
         ("weights", ctypes.c_void_p)]


class cptr_newton_stats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int32), ("linear_its", ctypes.c_int32),
                ("line_search_cuts", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("res0", ctypes.c_double), ("res", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double)]


class CptrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int32
_SIGS = {
    "cptr_default_options": (_I, [_P]),
    "cptr_create": (_I, [_P, _P]),
    "cptr_destroy": (None, [_P]),
    "cptr_last_error": (ctypes.c_char_p, [_P]),
    "cptr_setup": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _P, _I]),
    "cptr_solve": (_I, [_P, _P, _P, ctypes.c_double, _P, _I]),
    "cptr_apply_matrix": (_I, [_P, _P, _P]),
    "cptr_apply_weights": (_I, [_P, _P, _P]),
    "cptr_apply_stage1": (_I, [_P, _P, _P]),
    "cptr_apply_ilu": (_I, [_P, _P, _P]),
    "cptr_apply_precond": (_I, [_P, _P, _P]),
    "cptr_apply_ilu_static": (_I, [_P, _P, _P]),
    "cptr_apply_vcycle": (_I, [_P, _I, _P, _P]),
    "cptr_hierarchy_info": (_I, [_P, _I, _P, _P]),
    "cptr_hierarchy_level": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    "cptr_ilu_levels": (_I, [_P, _P, _P]),
    "cptr_launch_count": (ctypes.c_int64, []),
    "cptr_inject_wait_timeout": (_I, [_P, _I]),
    "cptr_set_profiling": (_I, [_P, ctypes.c_uint32]),
    "cptr_profile": (_I, [_P, _P, _P]),
    "cptr_profile_vcycle": (_I, [_P, _P, _P]),
    "cptr_set_partition": (_I, [_P, _I, _P, _I]),
    "cptr_setup_batch": (_I, [_P, _I, _I, _P, _P, _I]),
    "cptr_tuning": (_I, [_P, _P, _I, _P]),
    "cptr_solve_batch": (_I, [_P, _P, _P, ctypes.c_double, _P, _I]),
    "cptr_schur_features": (_I, [_P, _P, _I]),
    "cptr_mlp_loss_grad": (_I, [_P, _P, _P, _I, _P, _P, _P, _I]),
    "cptr_mlp_train": (_I, [_P, _P, _P, _I, _P, _I, ctypes.c_float, _P, _I]),
    "cptr_set_mlp": (_I, [_P, _P, _I]),
    "cptr_mlp_infer": (_I, [_P, _P, _I, _P, _I]),
    "cptr_schur_scaling": (_I, [_P, _P, _I]),
    "cptr_model_set": (_I, [_P, _P, _I]),
    "cptr_assemble": (_I, [_P, _P, _P, _P, _P, _P, _I]),
    "cptr_newton": (_I, [_P, _P, _P, ctypes.c_double, _I, _P, _I]),
}
PROFILE_FAMILIES = ("spmv", "stage1", "stage1_resid", "ilu", "arnoldi", "ilu_fwd", "ilu_bwd", "_7")
PROFILE_VCYCLE = tuple(f"{h}_{k}" for h in ("p", "T") for k in ("down", "restrict", "prolong", "post"))
PROFILE_MASK_VCYCLE = 1 << 7
SETUP_PHASES = {8: "setup_inputs", 9: "setup_amg_coarsen", 10: "setup_amg_rap", 11: "setup_amg_coarsest",
                12: "setup_ilu_host", 13: "setup_ilu_factor", 14: "setup_layout", 15: "setup_other"}


def select_library(variant: str = "") -> None:
    """Choose the library this process loads, before its first use: "" (libcptr.so) or "check"
    (libcptr_check.so, the bounds-checking build: every failed index check makes the call return
    CPTR_ECHECK)."""
    global LIB_PATH
    if _lib is not None:
        raise RuntimeError("the library is already loaded in this process")
    LIB_PATH = _build.VARIANTS[variant][0]


def load():
    """Load libcptr.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{os.path.basename(LIB_PATH)} not found at {LIB_PATH}: run __graft_entry__.build() "
                              "(no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def build(force: bool = False) -> str:
    return _build.build(force=force)


def _ptr(t):
    """Data pointer of a torch tensor or numpy array (None passes through)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _on_device(*ts):
    devs = {bool(getattr(t, "is_cuda", False)) for t in ts if t is not None}
    if len(devs) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return int(devs.pop()) if devs else 0


def _check(ctx, code, ok=(CPTR_OK,)):
    if code not in ok:
        msg = load().cptr_last_error(ctx)
        raise CptrError(code, msg.decode() if msg else "")
    return code


# ------------------------------------------------------------------------------------------------
# thin wrappers with the C names
def cptr_default_options(**kw) -> cptr_options:
    o = cptr_options()
    load().cptr_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "stage1" and isinstance(v, str):
            v = STAGE1[v]
        elif k == "stage2" and isinstance(v, str):
            v = STAGE2[v]
        elif k == "schur" and isinstance(v, str):
            v = SCHUR[v]
        elif k == "smoother" and isinstance(v, str):
            v = SMOOTHER[v]
        elif k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        elif k == "ilu_order" and isinstance(v, str):
            v = ILU_ORDER[v]
        elif k == "ilu_sweep" and isinstance(v, str):
            v = ILU_SWEEP[v]
        elif k == "decouple" and isinstance(v, str):
            v = DECOUPLE[v]
        setattr(o, k, v)
    return o


def cptr_create(opts: cptr_options) -> int:
    h = ctypes.c_void_p()
    code = load().cptr_create(ctypes.byref(h), ctypes.byref(opts))
    if code != CPTR_OK:
        raise CptrError(code, "cptr_create failed")
    return h.value


def cptr_destroy(ctx) -> None:
    load().cptr_destroy(ctx)


def cptr_setup(ctx, n_cells, b, row_ptr, col_idx, vals, unknown_kind, row_weights=None, st_vals=None):
    dev = _on_device(row_ptr, col_idx, vals, unknown_kind, row_weights, st_vals)
    return _check(ctx, load().cptr_setup(ctx, n_cells, b, _ptr(row_ptr), _ptr(col_idx), _ptr(vals),
                                         _ptr(unknown_kind), _ptr(row_weights), _ptr(st_vals), dev))


def cptr_solve(ctx, rhs, x, rtol):
    st = cptr_stats()
    dev = _on_device(rhs, x)
    code = _check(ctx, load().cptr_solve(ctx, _ptr(rhs), _ptr(x), rtol, ctypes.byref(st), dev),
                  ok=(CPTR_OK, CPTR_NOT_CONVERGED))
    return code, st


def _vec_call(name, ctx, *args):
    return _check(ctx, getattr(load(), name)(ctx, *args))


def cptr_apply_matrix(ctx, x, y):
    return _vec_call("cptr_apply_matrix", ctx, _ptr(x), _ptr(y))


def cptr_apply_weights(ctx, rhs, out):
    return _vec_call("cptr_apply_weights", ctx, _ptr(rhs), _ptr(out))


def cptr_apply_stage1(ctx, v, x1):
    return _vec_call("cptr_apply_stage1", ctx, _ptr(v), _ptr(x1))


def cptr_apply_ilu(ctx, r, z):
    return _vec_call("cptr_apply_ilu", ctx, _ptr(r), _ptr(z))


def cptr_apply_ilu_static(ctx, r, z):
    """Allocation-free ILU(0) application (scratch in a static device array, at most 2^20 unknowns)."""
    return _vec_call("cptr_apply_ilu_static", ctx, _ptr(r), _ptr(z))


def cptr_apply_precond(ctx, v, z):
    return _vec_call("cptr_apply_precond", ctx, _ptr(v), _ptr(z))


def cptr_apply_vcycle(ctx, which, b, x):
    return _vec_call("cptr_apply_vcycle", ctx, which, _ptr(b), _ptr(x))


def cptr_hierarchy_info(ctx, which):
    nlev = ctypes.c_int32()
    info = np.zeros(4 * 32, np.int32)
    _check(ctx, load().cptr_hierarchy_info(ctx, which, ctypes.byref(nlev), info.ctypes.data))
    return [dict(n=int(info[4 * l]), nnz=int(info[4 * l + 1]), nnzP=int(info[4 * l + 2]), dense=bool(info[4 * l + 3]))
            for l in range(nlev.value)]


def cptr_hierarchy_level(ctx, which, l, n, nnz, nnzP, coarse):
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(max(nnz, 1), np.int32)
    v = np.zeros(max(nnz, 1))
    dinv = np.zeros(max(n, 1))
    cf = np.zeros(n, np.int32) if not coarse else None
    Prp = np.zeros(n + 1, np.int32) if not coarse else None
    Pci = np.zeros(max(nnzP, 1), np.int32) if not coarse else None
    Pv = np.zeros(max(nnzP, 1)) if not coarse else None
    _check(ctx, load().cptr_hierarchy_level(ctx, which, l, _ptr(rp), _ptr(ci), _ptr(v), _ptr(dinv), _ptr(cf),
                                            _ptr(Prp), _ptr(Pci), _ptr(Pv)))
    out = dict(n=n, rp=rp, ci=ci[:nnz], v=v[:nnz], dinv=dinv[:n])
    if not coarse:
        out.update(cf=cf, Prp=Prp, Pci=Pci[:nnzP], Pv=Pv[:nnzP])
    return out


def cptr_ilu_levels(ctx):
    f, b = ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, load().cptr_ilu_levels(ctx, ctypes.byref(f), ctypes.byref(b)))
    return f.value, b.value


def cptr_launch_count() -> int:
    return int(load().cptr_launch_count())


def cptr_inject_wait_timeout(ctx, on: bool):
    return _check(ctx, load().cptr_inject_wait_timeout(ctx, int(bool(on))))


def cptr_set_profiling(ctx, mask: int):
    return _check(ctx, load().cptr_set_profiling(ctx, mask))


def cptr_profile(ctx):
    ms = np.zeros(16)
    cnt = np.zeros(16, np.int64)
    _check(ctx, load().cptr_profile(ctx, ms.ctypes.data, cnt.ctypes.data))
    out = {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(PROFILE_FAMILIES) if not name.startswith("_")}
    for i, name in SETUP_PHASES.items():
        out[name] = (float(ms[i]), int(cnt[i]))
    return out


def cptr_set_partition(ctx, part):
    """Part id per cell for the block-Jacobi ILU(0) (torch tensor or numpy array, int32); None removes it."""
    if part is None:
        return _check(ctx, load().cptr_set_partition(ctx, 0, None, 0))
    on = _on_device(part)
    if not on:
        part = np.ascontiguousarray(part, dtype=np.int32)
    return _check(ctx, load().cptr_set_partition(ctx, len(part), _ptr(part), int(on)))


def cptr_profile_vcycle(ctx):
    """{"p_down": (ms, launches), ...}: the finest level's V-cycle kernels of the last solve."""
    ms = np.zeros(8)
    cnt = np.zeros(8, np.int64)
    _check(ctx, load().cptr_profile_vcycle(ctx, ms.ctypes.data, cnt.ctypes.data))
    return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(PROFILE_VCYCLE)}


# ------------------------------------------------------------------------------------------------
def cptr_tuning(ctx):
    """Launch shapes in use: list of (hierarchy, level, kernel, lanes per row, threads per block)."""
    n = ctypes.c_int32(0)
    _check(ctx, load().cptr_tuning(ctx, None, 0, ctypes.byref(n)))
    rows = np.zeros((max(n.value, 1), 5), np.int32)
    _check(ctx, load().cptr_tuning(ctx, rows.ctypes.data, n.value, ctypes.byref(n)))
    return [tuple(int(v) for v in r) for r in rows[:n.value]]


def cptr_setup_batch(ctx, b, instances, unknown_kind):
    """instances: list of dicts with n_cells, row_ptr, col_idx, vals and optional row_weights,
    st_vals (all torch CUDA tensors or all numpy arrays)."""
    arr = (cptr_instance * len(instances))()
    arrays = [unknown_kind]
    for k, I in enumerate(instances):
        arr[k].n_cells = int(I["n_cells"])
        for f in ("row_ptr", "col_idx", "vals", "row_weights", "st_vals"):
            setattr(arr[k], f, _ptr(I.get(f)))
            arrays.append(I.get(f))
    dev = _on_device(*arrays)
    return _check(ctx, load().cptr_setup_batch(ctx, len(instances), b, arr, _ptr(unknown_kind), dev))


def cptr_solve_batch(ctx, rhs, x, rtol):
    """rhs, x: lists of per-instance arrays.  Returns (status code, list of cptr_stats)."""
    n = len(rhs)
    pr = (ctypes.c_void_p * n)(*[_ptr(r) for r in rhs])
    px = (ctypes.c_void_p * n)(*[_ptr(v) for v in x])
    st = (cptr_stats * n)()
    dev = _on_device(*rhs, *x)
    code = _check(ctx, load().cptr_solve_batch(ctx, pr, px, rtol, st, dev), ok=(CPTR_OK, CPTR_NOT_CONVERGED))
    return code, list(st)


def cptr_schur_features(ctx, feat):
    """feat: [n_cells, 16] float64 (torch CUDA tensor or numpy array), filled in place."""
    return _check(ctx, load().cptr_schur_features(ctx, _ptr(feat), _on_device(feat)))


def cptr_mlp_loss_grad(ctx, feat, target, params, grad):
    """Loss (returned) and gradient (into grad, float32) of the network at params."""
    loss = ctypes.c_double(0.0)
    dev = _on_device(feat, target, params, grad)
    _check(ctx, load().cptr_mlp_loss_grad(ctx, _ptr(feat), _ptr(target), int(feat.shape[0]), _ptr(params),
                                          _ptr(grad), ctypes.byref(loss), dev))
    return loss.value


def cptr_mlp_train(ctx, feat, target, params, steps, lr=1e-3):
    """Adam steps on params (float32, in place); returns the loss before each step."""
    hist = np.zeros(max(int(steps), 1))
    dev = _on_device(feat, target, params)
    _check(ctx, load().cptr_mlp_train(ctx, _ptr(feat), _ptr(target), int(feat.shape[0]), _ptr(params), int(steps),
                                      float(lr), hist.ctypes.data, dev))
    return hist[:int(steps)]


def cptr_set_mlp(ctx, params):
    return _check(ctx, load().cptr_set_mlp(ctx, _ptr(params), _on_device(params)))


def cptr_mlp_infer(ctx, feat, y):
    dev = _on_device(feat, y)
    return _check(ctx, load().cptr_mlp_infer(ctx, _ptr(feat), int(feat.shape[0]), _ptr(y), dev))


def cptr_schur_scaling(ctx, s):
    return _check(ctx, load().cptr_schur_scaling(ctx, _ptr(s), _on_device(s)))


_MODEL_ARRAYS = {"kh": np.float64, "kv": np.float64, "well_cell": np.int32, "well_kind": np.int32,
                 "well_a": np.float64, "well_c": np.float64, "heater_cell": np.int32, "heater_U": np.float64,
                 "heater_T": np.float64, "weights": np.float64}


def cptr_model_set(ctx, fields: dict):
    """Marshal a model description (scalars and arrays; arrays all host numpy or all torch CUDA)
    into cptr_model and hand it to the context."""
    m = cptr_model()
    keep = []
    arrays = [fields.get(k) for k in _MODEL_ARRAYS]
    on_dev = _on_device(*arrays)
    for k, dt in _MODEL_ARRAYS.items():
        a = fields.get(k)
        if a is None:
            continue
        if not on_dev:
            a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        count = a.numel() if hasattr(a, "numel") else a.size
        setattr(m, k, _ptr(a) if count else None)
    for k, t in cptr_model._fields_:
        if k in _MODEL_ARRAYS or k in ("n_wells", "n_heaters"):
            continue
        setattr(m, k, fields[k])
    m.n_wells = len(fields.get("well_cell", []))
    m.n_heaters = len(fields.get("heater_cell", []))
    return _check(ctx, load().cptr_model_set(ctx, ctypes.byref(m), on_dev))


def cptr_assemble(ctx, x, xn, R, J=None, Se=None):
    return _check(ctx, load().cptr_assemble(ctx, _ptr(x), _ptr(xn), _ptr(R), _ptr(J), _ptr(Se),
                                            _on_device(x, xn, R, J, Se)))


def cptr_newton(ctx, x, xn, rtol_lin, max_newton):
    st = cptr_newton_stats()
    code = _check(ctx, load().cptr_newton(ctx, _ptr(x), _ptr(xn), rtol_lin, max_newton, ctypes.byref(st),
                                          _on_device(x, xn)), ok=(CPTR_OK, CPTR_NOT_CONVERGED))
    return dict(status=STATUS.get(code, code), newton_its=st.newton_its, linear_its=st.linear_its,
                line_search_cuts=st.line_search_cuts, converged=bool(st.converged), res0=st.res0, res=st.res,
                setup_ms=st.setup_ms, solve_ms=st.solve_ms)


class Solver:
    """One CPTR-FGMRES context on the current CUDA device.

    ``Solver(stage1="full", restart=30, stream=torch.cuda.current_stream())`` then
    ``setup(...)`` with the BSR Jacobian and ``solve(rhs, rtol)``.  Arrays may be torch CUDA
    tensors (used in place) or host arrays (copied by the library).
    """

    def __init__(self, stream=None, **opts):
        s = getattr(stream, "cuda_stream", stream)
        self.opts = cptr_default_options(stream=s, **opts)
        self.ctx = cptr_create(self.opts)
        self.n = self.b = None
        self._keep = ()

    def close(self):
        if getattr(self, "ctx", None):
            cptr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def setup(self, n_cells, b, row_ptr, col_idx, vals, unknown_kind, row_weights=None, st_vals=None):
        self.n, self.b = int(n_cells), int(b)
        cptr_setup(self.ctx, self.n, self.b, row_ptr, col_idx, vals, unknown_kind, row_weights, st_vals)
        return self

    def solve(self, rhs, rtol=1e-6, x=None):
        import torch
        if x is None:
            x = torch.empty_like(rhs) if hasattr(rhs, "is_cuda") else np.zeros(self.n * self.b)
        code, st = cptr_solve(self.ctx, rhs, x, rtol)
        info = {f: getattr(st, f) for f, _ in cptr_stats._fields_}
        info["schur_used"] = SCHUR_NAMES.get(info["schur_used"], info["schur_used"])
        info["status"] = STATUS[code]
        return x, info

    def setup_batch(self, b, instances, unknown_kind):
        self.b = int(b)
        self.n_inst = [int(I["n_cells"]) for I in instances]
        cptr_setup_batch(self.ctx, self.b, instances, unknown_kind)
        return self

    def solve_batch(self, rhs, rtol=1e-6, x=None):
        import torch
        if x is None:
            x = [torch.empty_like(r) if hasattr(r, "is_cuda") else np.zeros(len(r)) for r in rhs]
        code, sts = cptr_solve_batch(self.ctx, rhs, x, rtol)
        infos = []
        for st in sts:
            info = {f: getattr(st, f) for f, _ in cptr_stats._fields_}
            info["schur_used"] = SCHUR_NAMES.get(info["schur_used"], info["schur_used"])
            infos.append(info)
        return x, STATUS[code], infos

    def hierarchy(self, which):
        levels = cptr_hierarchy_info(self.ctx, which)
        out = []
        for l, L in enumerate(levels):
            coarse = l == len(levels) - 1
            out.append(cptr_hierarchy_level(self.ctx, which, l, L["n"], L["nnz"], L["nnzP"], coarse))
            out[-1]["dense"] = L["dense"]
        return out
