"""Python binding of libdwos (ctypes).  Argument marshalling only: every step of
walk on spheres, differential walk on spheres and the estimator reductions runs
in the library's CUDA kernels.  PyTorch provides device memory and the stream.

The library must have been built (``paper_2405_12964_gb300.build.build()``);
there is no fallback: loading fails loudly when ``libdwos.so`` is missing or
no CUDA device is visible.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdwos.so")

MEM_HOST, MEM_DEVICE = 0, 1
KIND_SHELL, KIND_ROULETTE, KIND_CAPPED = 0, 1, 2

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "STEP_LIMIT", 5: "TIMEOUT",
          6: "NOT_IMPLEMENTED", 7: "STATE", 8: "OUTSIDE"}

RECORD_DTYPE = np.dtype([("u", "<f4"), ("elem", "<i4"), ("b1", "<f4"), ("b2", "<f4"),
                         ("c", "<f4", (3,)), ("meta", "<u4")])
DEBUG_DTYPE = np.dtype([("dudn", "<f4"), ("n", "<f4", (3,)), ("u_off", "<f4"), ("xbar", "<f4", (3,)),
                        ("u_plain", "<f4"), ("disp_n", "<f4"), ("disp_t", "<f4"), ("elem", "<i4")])


class Options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("h", ctypes.c_float), ("K", ctypes.c_int), ("B", ctypes.c_int),
                ("max_steps", ctypes.c_int), ("seed", ctypes.c_uint64), ("check_inside", ctypes.c_int),
                ("block_size", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("traversal", ctypes.c_int),
                ("dudn_estimator", ctypes.c_int)]


class RunStats(ctypes.Structure):
    _fields_ = [("steps_main", ctypes.c_uint64), ("steps_nested", ctypes.c_uint64), ("walks", ctypes.c_uint64),
                ("capped", ctypes.c_uint64), ("nodes_visited", ctypes.c_uint64), ("prims_tested", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("kernel_ms", ctypes.c_float), ("blocks", ctypes.c_int),
                ("wide_nodes_visited", ctypes.c_uint64)]


class DwosError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dwos {STATUS.get(status, status)}: {msg}")
        self.status = status


class BatchJob(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("n_query", ctypes.c_int), ("xq", ctypes.c_void_p),
                ("walks_per_point", ctypes.c_int), ("uref", ctypes.c_void_p), ("walk_id_base", ctypes.c_uint64),
                ("loss", ctypes.c_void_p), ("grad_param", ctypes.c_void_p), ("u_mean", ctypes.c_void_p)]


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_u64 = ctypes.c_uint64

# name -> argtypes (all entry points return int status unless noted)
_SIGS = {
    "dwos_create": [ctypes.POINTER(_vp), _i],
    "dwos_set_stream": [_vp, _vp],
    "dwos_sync": [_vp],
    "dwos_set_options": [_vp, ctypes.POINTER(Options)],
    "dwos_set_boundary": [_vp, _i, _i, _vp, _i, _vp, _i, _vp, _i],
    "dwos_set_params": [_vp, _vp, _i],
    "dwos_set_dirichlet_mapped": [_vp, _vp, _vp, _i],
    "dwos_set_dirichlet_field": [_vp, ctypes.POINTER(ctypes.c_double)],
    "dwos_set_pde": [_vp, ctypes.c_float, ctypes.c_float],
    "dwos_eval": [_vp, _i, _vp, _i, _vp, _vp, _vp, _vp, _i],
    "dwos_vjp": [_vp, _i, _vp, _vp, _i, _u64, _vp, _vp, _i],
    "dwos_grad_l2": [_vp, _i, _vp, _vp, _i, _u64, _vp, _vp, _vp, _i],
    "dwos_grad_l2_product": [_vp, _i, _vp, _vp, _i, _u64, _i, _vp, _vp, _vp, _i],
    "dwos_walk_records": [_vp, _i, _vp, _i, _u64, _i, _vp, _vp, _vp, _i],
    "dwos_last_stats": [_vp, ctypes.POINTER(RunStats)],
    "dwos_closest_point": [_vp, _i, _vp, _vp, _vp, _vp, _i],
    "dwos_closest_point_hint": [_vp, _i, _vp, _vp, _vp, _vp, _vp, _i],
    "dwos_inside": [_vp, _i, _vp, _vp, _i],
    "dwos_philox4x32_10": [_vp, _i, _vp, _vp, _vp, _i],
    "dwos_ball_weights": [_vp, _i, ctypes.c_float, _i, _vp, _vp, _vp, _vp, _i],
    "dwos_bessel_k0": [_vp, _i, _vp, _vp, _i],
    "dwos_bessel_k1": [_vp, _i, _vp, _vp, _i],
    "dwos_star_weight": [_vp, _i, ctypes.c_float, _i, _vp, _vp, _vp, _i],
    "dwos_set_neumann": [_vp, _vp, _i],
    "dwos_set_neumann_data": [_vp, _vp, _i],
    "dwos_eval_static": [_vp, _i, _vp, _i, _vp, _vp, _vp, _vp],
    "dwos_batch_create": [ctypes.POINTER(_vp), ctypes.POINTER(BatchJob), _i, _vp],
    "dwos_batch_run": [_vp],
    "dwos_batch_capture": [_vp],
    "dwos_batch_launch": [_vp],
    "dwos_batch_autotune": [_vp, _i],
    "dwos_batch_config": [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                          ctypes.POINTER(ctypes.c_float)],
    "dwos_batch_stats": [_vp, ctypes.POINTER(RunStats)],
    "dwos_batch_trace": [_vp, _i],
    "dwos_batch_records": [_vp, _i, _vp, _vp, _i],
    "dwos_grad_l2_cv": [_vp, _i, _vp, _vp, _i, _u64, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp],
    "dwos_mlp_create": [ctypes.POINTER(_vp), _i],
    "dwos_mlp_set_stream": [_vp, _vp],
    "dwos_mlp_set_params": [_vp, _vp, _i],
    "dwos_mlp_get_params": [_vp, _vp, _i],
    "dwos_mlp_loss_grad": [_vp, _i, _vp, _vp, _vp, _vp, _vp, _i],
    "dwos_mlp_train_step": [_vp, _i, _vp, _vp, _vp, ctypes.c_float, _vp, _i],
    "dwos_mlp_eval": [_vp, _i, _vp, _vp, _vp, _vp, _i],
    "dwos_mlp_sync": [_vp],
    "dwos_mlp_wait_probe": [_vp, _i],
    "dwos_set_traversal_budget": [_vp, _i],
    "dwos_cv_table": [_vp, _vp, _vp],
    "dwos_cv_training_set": [_vp, ctypes.c_longlong, _vp, _vp, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_float,
                             _vp, _vp, _vp, ctypes.POINTER(ctypes.c_longlong)],
    "dwos_bvh_info": [_vp, _vp],
    "dwos_probe_l2_read": [_i, ctypes.c_size_t, _i, _vp],
    "dwos_sample_domain": [_vp, _i, _vp, _vp, _u64, _vp, _vp, _vp],
    "dwos_grad_l2_weighted": [_vp, _i, _vp, _vp, _vp, _i, _u64, _vp, _vp, _vp, _i],
    "dwos_boundary_term_l2": [_vp, _vp, _vp, _vp, _vp, _i],
    "dwos_boundary_loss_l2": [_vp, _vp, _vp, _vp, _vp, _vp, _i],
    "dwos_get_vertices": [_vp, _vp, _i],
}
MLP_NPARAM = 14088


def lib():
    """Load libdwos.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2405_12964_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.dwos_destroy.argtypes = [_vp]
        L.dwos_destroy.restype = None
        L.dwos_last_error.argtypes = [_vp]
        L.dwos_last_error.restype = ctypes.c_char_p
        L.dwos_default_options.argtypes = [ctypes.POINTER(Options)]
        L.dwos_default_options.restype = None
        L.dwos_batch_destroy.argtypes = [_vp]
        L.dwos_batch_destroy.restype = None
        L.dwos_batch_last_error.argtypes = [_vp]
        L.dwos_batch_last_error.restype = ctypes.c_char_p
        L.dwos_mlp_destroy.argtypes = [_vp]
        L.dwos_mlp_destroy.restype = None
        L.dwos_mlp_last_error.argtypes = [_vp]
        L.dwos_mlp_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def exported_symbols():
    return sorted(list(_SIGS) + ["dwos_destroy", "dwos_last_error", "dwos_default_options", "dwos_batch_destroy",
                                 "dwos_batch_last_error", "dwos_mlp_destroy", "dwos_mlp_last_error"])


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Solver:
    """One library context on one CUDA device; all work on torch's current stream."""

    def __init__(self, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("dwos needs a CUDA device")
        self.device = torch.device("cuda", device)
        self._h = ctypes.c_void_p()
        L = lib()
        st = L.dwos_create(ctypes.byref(self._h), device)
        if st:
            raise DwosError(st, L.dwos_last_error(None).decode())
        self.dim = 0
        self.n_vert = 0
        self.n_param = 0
        self.opt = Options()
        L.dwos_default_options(ctypes.byref(self.opt))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib is not None:
            _lib.dwos_destroy(h)
            self._h = ctypes.c_void_p()

    # ---------------------------------------------------------------- plumbing
    def _check(self, st: int):
        if st:
            raise DwosError(st, lib().dwos_last_error(self._h).decode())

    def _stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        self._check(lib().dwos_set_stream(self._h, ctypes.c_void_p(s)))

    def _dev(self, a, dtype) -> torch.Tensor:
        return torch.as_tensor(np.asarray(a) if not torch.is_tensor(a) else a).to(
            device=self.device, dtype=dtype).contiguous()

    # ---------------------------------------------------------------- problem
    def set_options(self, **kw):
        for k, v in kw.items():
            if not hasattr(self.opt, k):
                raise KeyError(k)
            setattr(self.opt, k, v)
        self._check(lib().dwos_set_options(self._h, ctypes.byref(self.opt)))

    def set_boundary(self, vert, elem, jac=None):
        self._stream()
        v = self._dev(vert, torch.float32)
        e = self._dev(elem, torch.int32)
        j = None if jac is None else self._dev(jac, torch.float32)
        dim = v.shape[1]
        P = 0 if j is None else j.shape[2]
        self._check(lib().dwos_set_boundary(self._h, dim, v.shape[0], _ptr(v), e.shape[0], _ptr(e), P, _ptr(j),
                                            MEM_DEVICE))
        self.dim, self.n_vert, self.n_param, self.n_elem = dim, v.shape[0], P, e.shape[0]

    def set_params(self, theta):
        self._stream()
        t = self._dev(theta, torch.float32)
        self._check(lib().dwos_set_params(self._h, _ptr(t), MEM_DEVICE))

    def set_dirichlet_mapped(self, g, dg=None):
        self._stream()
        gt = self._dev(g, torch.float32)
        dgt = None if dg is None else self._dev(dg, torch.float32)
        self._check(lib().dwos_set_dirichlet_mapped(self._h, _ptr(gt), _ptr(dgt), MEM_DEVICE))

    def set_dirichlet_field(self, coeffs):
        c = (ctypes.c_double * 10)(*[float(x) for x in np.asarray(coeffs, dtype=np.float64).reshape(-1)[:10]])
        self._check(lib().dwos_set_dirichlet_field(self._h, c))

    def _per_element(self, a, dtype, tdtype):
        """One value per element of the current boundary, on the device (the C
        side reads n_elem of them)."""
        arr = a.reshape(-1) if torch.is_tensor(a) else np.asarray(a, dtype=dtype).reshape(-1)
        if arr.shape[0] != getattr(self, "n_elem", 0):
            raise ValueError(f"expected {getattr(self, 'n_elem', 0)} per-element values, got {arr.shape[0]}")
        return self._dev(arr, tdtype)

    def set_neumann(self, flags):
        """dwos_set_neumann: per-element flags, 1 = Neumann element (None: all Dirichlet)."""
        self._stream()
        ft = None if flags is None else self._per_element(flags, np.int32, torch.int32)
        self._check(lib().dwos_set_neumann(self._h, _ptr(ft), MEM_DEVICE))

    def set_neumann_data(self, h):
        """dwos_set_neumann_data: per-element Neumann data du/dn, n out of the domain (None: zero)."""
        self._stream()
        ht = None if h is None else self._per_element(h, np.float32, torch.float32)
        self._check(lib().dwos_set_neumann_data(self._h, _ptr(ht), MEM_DEVICE))

    def set_pde(self, sigma: float, f: float = 0.0):
        self._check(lib().dwos_set_pde(self._h, float(sigma), float(f)))

    def set_traversal_budget(self, max_fetches: int):
        """dwos_set_traversal_budget: node fetches one distance query may make (0: default)."""
        self._check(lib().dwos_set_traversal_budget(self._h, int(max_fetches)))

    def load_scene(self, sc, **opt):
        """Set boundary, data, PDE and the scene's eps / h / K / B / seed."""
        self.set_boundary(sc.vert, sc.elem, sc.jac)
        if getattr(sc, "neumann", None) is not None:
            self.set_neumann(sc.neumann)
        if getattr(sc, "neumann_h", None) is not None:
            self.set_neumann_data(sc.neumann_h)
        if sc.data == "field":
            self.set_dirichlet_field(sc.field)
        else:
            self.set_dirichlet_mapped(sc.g_vert, sc.dg_vert)
        self.set_pde(sc.sigma, sc.f)
        kw = dict(eps=sc.eps, h=sc.h, K=sc.K, B=sc.B, seed=sc.seed)
        kw.update(opt)
        self.set_options(**kw)

    # ---------------------------------------------------------------- estimators
    def eval(self, xq, walks: int, grad: bool = False):
        """u (and du/dtheta) at the query points: dict of FP64 device tensors."""
        self._stream()
        x = self._dev(xq, torch.float32)
        n = x.shape[0]
        dd = dict(device=self.device, dtype=torch.float64)
        u, se = torch.empty(n, **dd), torch.empty(n, **dd)
        du = dse = None
        if grad:
            du, dse = torch.empty(n, self.n_param, **dd), torch.empty(n, self.n_param, **dd)
        self._check(lib().dwos_eval(self._h, n, _ptr(x), int(walks), _ptr(u), _ptr(se), _ptr(du), _ptr(dse),
                                    MEM_DEVICE))
        out = {"u": u, "u_se": se}
        if grad:
            out.update(du=du, du_se=dse)
        return out

    def vjp(self, xq, w, walks: int, walk_id_base: int = 1 << 40, vertex_grad: bool = False):
        self._stream()
        x = self._dev(xq, torch.float32)
        wt = self._dev(w, torch.float32)
        dd = dict(device=self.device, dtype=torch.float64)
        g = torch.empty(max(self.n_param, 1), **dd)
        gv = torch.empty(self.n_vert, self.dim, **dd) if vertex_grad else None
        self._check(lib().dwos_vjp(self._h, x.shape[0], _ptr(x), _ptr(wt), int(walks), int(walk_id_base), _ptr(g),
                                   _ptr(gv), MEM_DEVICE))
        return (g[:self.n_param], gv) if vertex_grad else g[:self.n_param]

    def grad_l2(self, xq, uref, walks: int, walk_id_base: int = 0, vertex_grad: bool = False):
        self._stream()
        x = self._dev(xq, torch.float32)
        ur = self._dev(uref, torch.float32)
        dd = dict(device=self.device, dtype=torch.float64)
        loss = torch.empty(1, **dd)
        g = torch.empty(max(self.n_param, 1), **dd)
        gv = torch.empty(self.n_vert, self.dim, **dd) if vertex_grad else None
        self._check(lib().dwos_grad_l2(self._h, x.shape[0], _ptr(x), _ptr(ur), int(walks), int(walk_id_base),
                                       _ptr(loss), _ptr(g), _ptr(gv), MEM_DEVICE))
        return (loss, g[:self.n_param], gv) if vertex_grad else (loss, g[:self.n_param])

    def grad_l2_product(self, xq, uref, walks: int, product: str = "ustat", walk_id_base: int = 0):
        """dwos_grad_l2_product: the squared-loss gradient with the U-statistic
        ("ustat"), correlated ("correlated") or uncorrelated ("uncorrelated")
        product estimator.  Returns (loss, grad) as device FP64 tensors."""
        code = {"ustat": 0, "correlated": 1, "uncorrelated": 2}[product]
        self._stream()
        x = self._dev(xq, torch.float32)
        u = self._dev(uref, torch.float32)
        loss = torch.empty(1, device=self.device, dtype=torch.float64)
        g = torch.empty(max(self.n_param, 1), device=self.device, dtype=torch.float64)
        self._check(lib().dwos_grad_l2_product(self._h, x.shape[0], _ptr(x), _ptr(u), int(walks), int(walk_id_base),
                                               code, _ptr(loss), _ptr(g), None, MEM_DEVICE))
        return loss, g[:self.n_param]

    def grad_l2_cv(self, xq, uref, walks: int, walk_id_base: int = 0, cv_grad=None, whole_walk: bool = False,
                   cv_elem=None, samples: bool = False, debug: bool = False):
        """dwos_grad_l2_cv: loss, gradient, per-point SE of u without / with the
        control variate, and optionally the training samples and debug records."""
        self._stream()
        x = self._dev(xq, torch.float32)
        ur = self._dev(uref, torch.float32)
        n = x.shape[0]
        cg = None if cv_grad is None else self._dev(cv_grad, torch.float32)
        cq = None
        if cv_elem is not None:
            cq = self._dev(cv_elem, torch.float32)
            if cq.dim() != 2 or cq.shape[1] != 4:
                raise ValueError("cv_elem must be (n_elem, 4): du/dn surrogate and tangential gradient")
        dd = dict(device=self.device, dtype=torch.float64)
        loss = torch.empty(1, **dd)
        g = torch.empty(max(self.n_param, 1), **dd)
        se = torch.empty(2, n, **dd)
        smp = torch.empty(n * int(walks), 4, device=self.device, dtype=torch.float32) if samples else None
        dbg = torch.empty(n * int(walks) * DEBUG_DTYPE.itemsize, device=self.device, dtype=torch.uint8) if debug else None
        self._check(lib().dwos_grad_l2_cv(self._h, n, _ptr(x), _ptr(ur), int(walks), int(walk_id_base), _ptr(cg),
                                          1 if whole_walk else 0, _ptr(cq), _ptr(smp), _ptr(dbg), _ptr(loss), _ptr(g),
                                          _ptr(se)))
        out = {"loss": loss, "grad": g[:self.n_param], "u_se": se[0], "u_se_cv": se[1]}
        if samples:
            out["samples"] = smp
        if debug:
            out["debug"] = dbg
        return out

    # ------------------------------------------------ volume-integrated functional
    def sample_domain(self, n_try: int, box_lo, box_hi, seed: int = 0):
        """Points sampled uniformly in the box and kept inside Omega (dwos_sample_domain):
        (points on the device, the quadrature weight each carries)."""
        self._stream()
        pts = torch.empty(n_try, self.dim, device=self.device, dtype=torch.float32)
        lo = (ctypes.c_float * 3)(*[float(v) for v in box_lo])
        hi = (ctypes.c_float * 3)(*[float(v) for v in box_hi])
        n_in = ctypes.c_int()
        w = ctypes.c_float()
        self._check(lib().dwos_sample_domain(self._h, int(n_try), lo, hi, int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(pts),
                                             ctypes.byref(n_in), ctypes.byref(w)))
        return pts[:n_in.value], float(w.value)

    def grad_l2_weighted(self, xq, uref, weight, walks: int, walk_id_base: int = 0):
        """dwos_grad_l2_weighted: loss sum_p w_p 1/2 (u_p - uref_p)^2 and its gradient."""
        self._stream()
        x = self._dev(xq, torch.float32)
        u = self._dev(uref, torch.float32)
        w = self._dev(weight, torch.float32)
        loss = torch.empty(1, device=self.device, dtype=torch.float64)
        g = torch.empty(max(self.n_param, 1), device=self.device, dtype=torch.float64)
        self._check(lib().dwos_grad_l2_weighted(self._h, x.shape[0], _ptr(x), _ptr(u), _ptr(w), int(walks),
                                                int(walk_id_base), _ptr(loss), _ptr(g), None, MEM_DEVICE))
        return loss, g[:self.n_param]

    def boundary_term_l2(self, box_lo, box_hi, uref_vert=None):
        """dwos_boundary_term_l2: int_Gamma M V_n 1/2 (g - uref)^2 dA per parameter (numpy)."""
        self._stream()
        lo = (ctypes.c_float * 3)(*[float(v) for v in box_lo])
        hi = (ctypes.c_float * 3)(*[float(v) for v in box_hi])
        ur = None if uref_vert is None else self._dev(uref_vert, torch.float32)
        g = torch.empty(max(self.n_param, 1), device=self.device, dtype=torch.float64)
        self._check(lib().dwos_boundary_term_l2(self._h, lo, hi, _ptr(ur), _ptr(g), MEM_DEVICE))
        return g[:self.n_param].cpu().numpy()

    def boundary_loss_l2(self, box_lo, box_hi, ub_vert=None):
        """dwos_boundary_loss_l2: (J_b, dJ_b/dtheta) of int_Gamma m 1/2 (g - ub)^2 dA (numpy)."""
        self._stream()
        lo = (ctypes.c_float * 3)(*[float(v) for v in box_lo])
        hi = (ctypes.c_float * 3)(*[float(v) for v in box_hi])
        ub = None if ub_vert is None else self._dev(ub_vert, torch.float32)
        loss = torch.empty(1, device=self.device, dtype=torch.float64)
        g = torch.empty(max(self.n_param, 1), device=self.device, dtype=torch.float64)
        self._check(lib().dwos_boundary_loss_l2(self._h, lo, hi, _ptr(ub), _ptr(loss), _ptr(g), MEM_DEVICE))
        return float(loss.cpu()[0]), g[:self.n_param].cpu().numpy()

    def general_functional_gradient(self, box_lo, box_hi, uref_fn, walks: int, n_try: int, bbox_lo, bbox_hi,
                                    ub_vert=None, seed: int = 0, walk_id_base: int = 0):
        """Eq. (general_functional_deriv): the volume part of functional_gradient (mask box
        box_lo / box_hi, target uref_fn) plus the boundary loss int_Gamma m 1/2 (g - ub)^2 dA
        with m the box bbox_lo / bbox_hi and ub per vertex.  Returns (J estimate, dJ/dtheta)."""
        jv, gv = self.functional_gradient(box_lo, box_hi, uref_fn, walks, n_try, seed, walk_id_base)
        jb, gb = self.boundary_loss_l2(bbox_lo, bbox_hi, ub_vert)
        return jv + jb, gv + gb

    def functional_gradient(self, box_lo, box_hi, uref_fn, walks: int, n_try: int, seed: int = 0,
                            walk_id_base: int = 0):
        """Eq. (functional_deriv) for J = int_Omega M 1/2 (u - uref)^2 with M the box:
        the domain term from points sampled in the box (uref_fn maps an (n, dim)
        numpy array to uref there) plus the boundary term with uref_fn at the
        vertices.  Returns (J estimate, dJ/dtheta) as numpy."""
        pts, w = self.sample_domain(n_try, box_lo, box_hi, seed)
        p = pts.cpu().numpy().astype(np.float64)
        ur = np.asarray(uref_fn(p), dtype=np.float32).reshape(-1)
        loss, g = self.grad_l2_weighted(pts, ur, np.full(len(p), w, np.float32), walks, walk_id_base)
        vert = self.current_vertices()
        gb = self.boundary_term_l2(box_lo, box_hi, np.asarray(uref_fn(vert), np.float32).reshape(-1))
        return float(loss.cpu()[0]), g.cpu().numpy() + gb

    def current_vertices(self) -> np.ndarray:
        """Vertex positions at the current parameters (dwos_get_vertices)."""
        out = np.empty((self.n_vert, self.dim), dtype=np.float32)
        self._check(lib().dwos_get_vertices(self._h, out.ctypes.data_as(ctypes.c_void_p), MEM_HOST))
        return out.astype(np.float64)

    def bvh_info(self) -> dict:
        info = (ctypes.c_int32 * 6)()
        self._check(lib().dwos_bvh_info(self._h, info))
        keys = ("n_elem", "n_tree", "n_big", "n_internal", "n_wide", "wide_depth")
        return dict(zip(keys, [int(v) for v in info]))

    def cv_table(self, net: "ControlVariateNet") -> torch.Tensor:
        """The nested walks' control-variate table (n_elem, 4) on the device:
        the network's du/dn head at each element's centre and the data's
        tangential gradient (dwos_cv_table)."""
        self._stream()
        out = torch.empty(self.n_elem, 4, device=self.device, dtype=torch.float32)
        self._check(lib().dwos_cv_table(self._h, net._h, _ptr(out)))
        return out

    def cv_training_set(self, samples: torch.Tensor, debug: Optional[torch.Tensor], stride: int, offset: int,
                        q_weight: float):
        """dwos_cv_training_set: (x, target, mask) device tensors of the network's
        training rows from a grad_l2_cv call's samples / debug records."""
        self._stream()
        n = samples.shape[0]
        rows = (n - offset + stride - 1) // stride * (2 if debug is not None else 1)
        x = torch.empty(rows, 2, device=self.device, dtype=torch.float32)
        t = torch.empty(rows, 2, device=self.device, dtype=torch.float32)
        m = torch.empty(rows, 2, device=self.device, dtype=torch.float32)
        got = ctypes.c_longlong()
        self._check(lib().dwos_cv_training_set(self._h, n, _ptr(samples), _ptr(debug), int(stride), int(offset),
                                               float(q_weight), _ptr(x), _ptr(t), _ptr(m), ctypes.byref(got)))
        assert got.value == rows
        return x, t, m

    def walk_records(self, xq, walks: int, walk_id_base: int = 0, differential: bool = True,
                     trace: bool = False, debug: bool = False):
        """Per-walk records as numpy structured arrays (row p * walks + w)."""
        self._stream()
        x = self._dev(xq, torch.float32)
        n = x.shape[0] * int(walks)
        rec = torch.empty(n * 32, device=self.device, dtype=torch.uint8)
        K1 = self.opt.K + 1
        tr = torch.empty(n * K1, device=self.device, dtype=torch.int32) if trace else None
        db = torch.empty(n * DEBUG_DTYPE.itemsize, device=self.device, dtype=torch.uint8) if debug else None
        self._check(lib().dwos_walk_records(self._h, x.shape[0], _ptr(x), int(walks), int(walk_id_base),
                                            1 if differential else 0, _ptr(rec), _ptr(tr), _ptr(db), MEM_DEVICE))
        self.sync()
        out = {"rec": rec.cpu().numpy().view(RECORD_DTYPE)}
        if trace:
            out["trace"] = tr.cpu().numpy().view(np.uint32).reshape(n, K1)
        if debug:
            out["debug"] = db.cpu().numpy().view(DEBUG_DTYPE)
        return out

    def sync(self):
        self._check(lib().dwos_sync(self._h))

    def stats(self) -> dict:
        s = RunStats()
        self._check(lib().dwos_last_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in RunStats._fields_}

    # ---------------------------------------------------------------- queries
    def closest_point(self, p):
        self._stream()
        x = self._dev(p, torch.float32)
        n = x.shape[0]
        d = torch.empty(n, device=self.device, dtype=torch.float32)
        e = torch.empty(n, device=self.device, dtype=torch.int32)
        b = torch.empty(n, 2, device=self.device, dtype=torch.float32)
        self._check(lib().dwos_closest_point(self._h, n, _ptr(x), _ptr(d), _ptr(e), _ptr(b), MEM_DEVICE))
        return d, e, b

    def closest_point_hint(self, p, hint_elem):
        self._stream()
        x = self._dev(p, torch.float32)
        h = self._dev(hint_elem, torch.int32)
        n = x.shape[0]
        d = torch.empty(n, device=self.device, dtype=torch.float32)
        e = torch.empty(n, device=self.device, dtype=torch.int32)
        b = torch.empty(n, 2, device=self.device, dtype=torch.float32)
        self._check(lib().dwos_closest_point_hint(self._h, n, _ptr(x), _ptr(h), _ptr(d), _ptr(e), _ptr(b),
                                                  MEM_DEVICE))
        return d, e, b

    def inside(self, p):
        self._stream()
        x = self._dev(p, torch.float32)
        out = torch.empty(x.shape[0], device=self.device, dtype=torch.int32)
        self._check(lib().dwos_inside(self._h, x.shape[0], _ptr(x), _ptr(out), MEM_DEVICE))
        return out

    def philox(self, ctr, key):
        self._stream()
        c = torch.as_tensor(np.asarray(ctr, dtype=np.uint32).view(np.int32)).to(self.device).contiguous()
        k = torch.as_tensor(np.asarray(key, dtype=np.uint32).view(np.int32)).to(self.device).contiguous()
        n = c.numel() // 4
        out = torch.empty(n * 4, device=self.device, dtype=torch.int32)
        self._check(lib().dwos_philox4x32_10(self._h, n, _ptr(c), _ptr(k), _ptr(out), MEM_DEVICE))
        return out.cpu().numpy().view(np.uint32).reshape(n, 4)

    def ball_weights(self, dim: int, sigma: float, d, u):
        """(source factor |B(d)| G_d(r), recursive weight alpha) per (d, u) pair,
        as the walk kernel evaluates them (dwos_ball_weights); numpy float32."""
        self._stream()
        dt = self._dev(d, torch.float32)
        ut = self._dev(u, torch.float32)
        n = dt.numel()
        src = torch.empty(n, device=self.device, dtype=torch.float32)
        al = torch.empty(n, device=self.device, dtype=torch.float32)
        self._check(lib().dwos_ball_weights(self._h, int(dim), float(sigma), n, _ptr(dt), _ptr(ut), _ptr(src),
                                            _ptr(al), MEM_DEVICE))
        return src.cpu().numpy(), al.cpu().numpy()

    def bessel_k0(self, x):
        """K0(x) as the 2D source weight evaluates it (dwos_bessel_k0); numpy float32."""
        return self._bessel(lib().dwos_bessel_k0, x)

    def bessel_k1(self, x):
        """K1(x) as the walk-on-stars step weight evaluates it (dwos_bessel_k1); numpy float32."""
        return self._bessel(lib().dwos_bessel_k1, x)

    def _bessel(self, fn, x):
        self._stream()
        xt = self._dev(x, torch.float32)
        out = torch.empty(xt.numel(), device=self.device, dtype=torch.float32)
        self._check(fn(self._h, xt.numel(), _ptr(xt), _ptr(out), MEM_DEVICE))
        return out.cpu().numpy()

    def star_weight(self, dim: int, sigma: float, t, R):
        """The walk-on-stars step's survival weight (dwos_star_weight); numpy float32."""
        self._stream()
        tt, Rt = self._dev(t, torch.float32), self._dev(R, torch.float32)
        out = torch.empty(tt.numel(), device=self.device, dtype=torch.float32)
        self._check(lib().dwos_star_weight(self._h, int(dim), float(sigma), tt.numel(), _ptr(tt), _ptr(Rt), _ptr(out),
                                           MEM_DEVICE))
        return out.cpu().numpy()


class Batch:
    """Many reverse-mode problems in one pass (dwos_batch_*): each job is
    (solver, xq, walks_per_point, uref, walk_id_base).  Outputs per job:
    loss (1), grad (n_param), u_mean (n_query), FP64 device tensors.  All work
    runs on the batch's own CUDA stream (`self.stream`)."""

    def __init__(self, jobs, device: int = 0):
        self.device = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=self.device)
        self.solvers, self.keep, self.out, self.walks = [], [], [], []
        arr = (BatchJob * len(jobs))()
        for k, (solver, xq, walks, uref, base) in enumerate(jobs):
            x = solver._dev(xq, torch.float32)
            ur = solver._dev(uref, torch.float32)
            dd = dict(device=self.device, dtype=torch.float64)
            o = {"loss": torch.zeros(1, **dd), "grad": torch.zeros(max(solver.n_param, 1), **dd),
                 "u_mean": torch.zeros(x.shape[0], **dd)}
            self.solvers.append(solver)
            self.walks.append(int(walks))
            self.keep += [x, ur]
            self.out.append(o)
            arr[k] = BatchJob(solver._h.value, x.shape[0], x.data_ptr(), int(walks), ur.data_ptr(), int(base),
                              o["loss"].data_ptr(), o["grad"].data_ptr(), o["u_mean"].data_ptr())
        torch.cuda.synchronize(self.device)
        self._h = ctypes.c_void_p()
        st = lib().dwos_batch_create(ctypes.byref(self._h), arr, len(jobs), ctypes.c_void_p(self.stream.cuda_stream))
        if st:
            raise DwosError(st, lib().dwos_batch_last_error(None).decode())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib is not None:
            _lib.dwos_batch_destroy(h)
            self._h = ctypes.c_void_p()

    def _check(self, st):
        if st:
            raise DwosError(st, lib().dwos_batch_last_error(self._h).decode())

    def run(self):
        self._check(lib().dwos_batch_run(self._h))

    def capture(self):
        self._check(lib().dwos_batch_capture(self._h))

    def launch(self):
        self._check(lib().dwos_batch_launch(self._h))

    def autotune(self, reps: int = 2):
        self._check(lib().dwos_batch_autotune(self._h, int(reps)))

    def config(self, dim: int) -> dict:
        bs, per, tr, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        self._check(lib().dwos_batch_config(self._h, dim, ctypes.byref(bs), ctypes.byref(per), ctypes.byref(tr),
                                            ctypes.byref(ms)))
        return {"block_size": bs.value, "blocks_per_sm": per.value, "traversal": tr.value, "walk_ms": ms.value}

    def stats(self) -> dict:
        s = RunStats()
        self._check(lib().dwos_batch_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in RunStats._fields_}

    def synchronize(self):
        self.stream.synchronize()

    def trace(self, enable: bool = True):
        """dwos_batch_trace: write per-walk traces in later passes."""
        self._check(lib().dwos_batch_trace(self._h, 1 if enable else 0))

    def records(self, job: int, trace: bool = False):
        """Records (numpy RECORD_DTYPE, row p * W + w) and optionally traces ((K + 1) uint32
        per walk) of job `job` from the last pass (dwos_batch_records)."""
        sv = self.solvers[job]
        n = int(self.keep[2 * job].shape[0]) * int(self.walks[job])
        rec = np.empty(n, dtype=RECORD_DTYPE)
        K1 = sv.opt.K + 1
        tr = np.empty(n * K1, dtype=np.uint32) if trace else None
        self._check(lib().dwos_batch_records(self._h, int(job), rec.ctypes.data_as(ctypes.c_void_p),
                                             None if tr is None else tr.ctypes.data_as(ctypes.c_void_p), MEM_HOST))
        return (rec, tr.reshape(n, K1)) if trace else rec

    def results(self):
        self.synchronize()
        return [{"loss": float(o["loss"][0]), "grad": o["grad"][:sv.n_param].cpu().numpy(),
                 "u_mean": o["u_mean"].cpu().numpy()} for o, sv in zip(self.out, self.solvers)]


class ControlVariateNet:
    """The control-variate network (dwos_mlp_*): 5 features -> 4 x 64 tanh ->
    outputs (u, du/dn); trained and evaluated with the library's tcgen05
    tensor-core kernel."""

    def __init__(self, device: int = 0, params=None, seed: int = 0):
        self.device = torch.device("cuda", device)
        self._h = ctypes.c_void_p()
        st = lib().dwos_mlp_create(ctypes.byref(self._h), device)
        if st:
            raise DwosError(st, lib().dwos_mlp_last_error(None).decode())
        if params is None:
            params = init_mlp_params(seed)
        self.set_params(params)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib is not None:
            _lib.dwos_mlp_destroy(h)
            self._h = ctypes.c_void_p()

    def _check(self, st):
        if st:
            raise DwosError(st, lib().dwos_mlp_last_error(self._h).decode())

    def _stream(self):
        self._check(lib().dwos_mlp_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)))

    def _dev(self, a, dtype=torch.float32):
        return torch.as_tensor(np.asarray(a) if not torch.is_tensor(a) else a).to(device=self.device,
                                                                                     dtype=dtype).contiguous()

    def set_params(self, p):
        self._stream()
        t = self._dev(p)
        self._check(lib().dwos_mlp_set_params(self._h, _ptr(t), MEM_DEVICE))
        torch.cuda.synchronize(self.device)

    def sync(self):
        """Wait for queued work; raises if a tensor-core product timed out."""
        self._stream()
        self._check(lib().dwos_mlp_sync(self._h))

    def wait_probe(self, polls: int):
        """dwos_mlp_wait_probe: a bounded wait that runs out (raises DwosError TIMEOUT)."""
        self._stream()
        self._check(lib().dwos_mlp_wait_probe(self._h, int(polls)))

    def params(self):
        self._stream()
        out = torch.empty(MLP_NPARAM, device=self.device, dtype=torch.float32)
        self._check(lib().dwos_mlp_get_params(self._h, _ptr(out), MEM_DEVICE))
        return out

    def loss_grad(self, x, target, mask):
        self._stream()
        x, t, m = self._dev(x), self._dev(target), self._dev(mask)
        g = torch.empty(MLP_NPARAM, device=self.device, dtype=torch.float32)
        loss = torch.empty(1, device=self.device, dtype=torch.float64)
        self._check(lib().dwos_mlp_loss_grad(self._h, x.shape[0], _ptr(x), _ptr(t), _ptr(m), _ptr(g), _ptr(loss),
                                             MEM_DEVICE))
        return loss, g

    def train_step(self, x, target, mask, lr: float = 1e-3):
        self._stream()
        x, t, m = self._dev(x), self._dev(target), self._dev(mask)
        loss = torch.empty(1, device=self.device, dtype=torch.float64)
        self._check(lib().dwos_mlp_train_step(self._h, x.shape[0], _ptr(x), _ptr(t), _ptr(m), float(lr), _ptr(loss),
                                              MEM_DEVICE))
        return loss

    def eval(self, x):
        self._stream()
        x = self._dev(x)
        n = x.shape[0]
        u = torch.empty(n, device=self.device, dtype=torch.float32)
        gu = torch.empty(n, 2, device=self.device, dtype=torch.float32)
        q = torch.empty(n, device=self.device, dtype=torch.float32)
        self._check(lib().dwos_mlp_eval(self._h, n, _ptr(x), _ptr(u), _ptr(gu), _ptr(q), MEM_DEVICE))
        return u, gu, q


def probe_l2_read(device: int = 0, nbytes: int = 32 << 20, reps: int = 50) -> float:
    """Measured read bandwidth (GB/s) of an L2-resident buffer (dwos_probe_l2_read)."""
    out = ctypes.c_double()
    st = lib().dwos_probe_l2_read(device, nbytes, reps, ctypes.byref(out))
    if st:
        raise DwosError(st, lib().dwos_last_error(None).decode())
    return out.value


def init_mlp_params(seed: int = 0) -> np.ndarray:
    """Xavier-uniform weights (unused input columns and output rows zero), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in, used_in, used_out in [(64, 16, 5, 64), (64, 64, 64, 64), (64, 64, 64, 64),
                                               (64, 64, 64, 64), (8, 64, 64, 2)]:
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        w = rng.uniform(-lim, lim, size=(fan_out, fan_in))
        w[:, used_in:] = 0.0
        w[used_out:, :] = 0.0
        parts += [w.reshape(-1), np.zeros(fan_out)]
    return np.concatenate(parts).astype(np.float32)


class DWoSFunction(torch.autograd.Function):
    """u(theta) at fixed query points, with the adjoint through differential walks.

    forward(theta): v = v_ref + J theta, BVH rebuild, walk on spheres (Algorithm 1)
    backward(grad_u): grad_theta = sum_p grad_u[p] E[udot_p] from differential
    walks (Algorithm 2) drawn with walk ids disjoint from the forward's, so the
    product with a cotangent built from the forward output stays uncorrelated
    (Sec. 4.3, Eq. uncorrelated_product); scatter + adjoint GEMV in the library.
    """

    @staticmethod
    def forward(ctx, theta, solver: Solver, xq, walks: int, backward_walks: int, backward_base: int):
        solver.set_params(theta.detach())
        out = solver.eval(xq, walks)
        ctx.solver = solver
        ctx.xq = xq
        ctx.bw = backward_walks
        ctx.base = backward_base
        ctx.save_for_backward(theta.detach().clone())
        return out["u"].to(dtype=theta.dtype)     # on the solver's device

    @staticmethod
    def backward(ctx, grad_u):
        (theta,) = ctx.saved_tensors
        s = ctx.solver
        s.set_params(theta)
        g = s.vjp(ctx.xq, grad_u.detach().to(torch.float32), ctx.bw, walk_id_base=ctx.base)
        return g.to(device=theta.device, dtype=theta.dtype), None, None, None, None, None


def solve(theta, solver: Solver, xq, walks: int, backward_walks: Optional[int] = None,
          backward_base: int = 1 << 40):
    """Differentiable u(theta) at xq (see DWoSFunction)."""
    return DWoSFunction.apply(theta, solver, xq, walks, backward_walks or walks, backward_base)
