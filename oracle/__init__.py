"""FP64 CPU oracle for Differential Walk on Spheres (Miller et al., TOG 2024).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It never imports the
CUDA library's package and shares no code with it; both sides receive the same
seeded scenes from a generator module that contains none of the method's
arithmetic.

Contents
  oracle.cpp       Algorithms 1 and 2 in FP64 with brute-force closest point and
                   an independent Philox4x32-10 (ctypes-loaded from liboracle.so);
                   walks on stars for mixed Dirichlet / Neumann boundaries (Sec.
                   3.4, 4.2), reflecting or with Neumann data du/dn
  estimators.py    per-point means, the product estimators of Sec. 4.3, VJPs
  closed_forms.py  exact solutions used to pin the oracle (disk, ball, and the
                   mixed-boundary scenes: quarter disk, strips, cube, cylinder
                   and sphere flow, boxes and an annulus with Neumann data)
  cv.py            the nested walks' control-variate table (tangential data gradient)
  mlp.py           the control-variate network with BF16 product operands, and
                   error bounds for an FP32-accumulating implementation
  functional.py    the volume-integrated and boundary shape functionals
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field as dc_field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++, OpenMP, no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n_vert", ctypes.c_int),
        ("vert", ctypes.POINTER(ctypes.c_double)),
        ("n_elem", ctypes.c_int),
        ("elem", ctypes.POINTER(ctypes.c_int)),
        ("n_param", ctypes.c_int),
        ("jac", ctypes.POINTER(ctypes.c_double)),
        ("data_kind", ctypes.c_int),
        ("g_vert", ctypes.POINTER(ctypes.c_double)),
        ("dg_vert", ctypes.POINTER(ctypes.c_double)),
        ("field_kind", ctypes.c_int),
        ("field", ctypes.c_double * 10),
        ("sigma", ctypes.c_double),
        ("f", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("h", ctypes.c_double),
        ("K", ctypes.c_int),
        ("max_steps", ctypes.c_int),
        ("seed_lo", ctypes.c_uint32),
        ("seed_hi", ctypes.c_uint32),
        ("cv_elem", ctypes.POINTER(ctypes.c_double)),
        ("dudn_mode", ctypes.c_int),
        ("neumann", ctypes.POINTER(ctypes.c_int)),
        ("neumann_h", ctypes.POINTER(ctypes.c_double)),
    ]


class _WalkOut(ctypes.Structure):
    _fields_ = [
        ("u_hat", ctypes.POINTER(ctypes.c_double)),
        ("udot", ctypes.POINTER(ctypes.c_double)),
        ("dudn", ctypes.POINTER(ctypes.c_double)),
        ("u_off", ctypes.POINTER(ctypes.c_double)),
        ("elem", ctypes.POINTER(ctypes.c_int)),
        ("bary", ctypes.POINTER(ctypes.c_double)),
        ("normal", ctypes.POINTER(ctypes.c_double)),
        ("xbar", ctypes.POINTER(ctypes.c_double)),
        ("kind", ctypes.POINTER(ctypes.c_int)),
        ("steps", ctypes.POINTER(ctypes.c_int)),
        ("x1", ctypes.POINTER(ctypes.c_double)),
        ("x_end", ctypes.POINTER(ctypes.c_double)),
        ("u_plain", ctypes.POINTER(ctypes.c_double)),
        ("disp_n", ctypes.POINTER(ctypes.c_double)),
        ("disp_t", ctypes.POINTER(ctypes.c_double)),
    ]


KIND_SHELL, KIND_ROULETTE, KIND_CAPPED = 0, 1, 2


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            up = ctypes.POINTER(ctypes.c_uint32)
            L.oracle_philox4x32_10.argtypes = [up, up, up]
            L.oracle_philox4x32_10.restype = None
            L.oracle_uniform.argtypes = [ctypes.c_uint32]
            L.oracle_uniform.restype = ctypes.c_double
            L.oracle_alpha.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
            L.oracle_alpha.restype = ctypes.c_double
            L.oracle_source_weight.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double]
            L.oracle_source_weight.restype = ctypes.c_double
            L.oracle_star_weight.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.oracle_star_weight.restype = ctypes.c_double
            L.oracle_turn_inward.argtypes = [ctypes.c_int, dp, dp, dp]
            L.oracle_turn_inward.restype = None
            L.oracle_ray_neumann.argtypes = [ctypes.POINTER(_Scene), dp, dp, ctypes.c_double, ctypes.c_int, dp,
                                             ctypes.c_int, dp, ip]
            L.oracle_ray_neumann.restype = ctypes.c_double
            L.oracle_neumann_data_sample.argtypes = [ctypes.POINTER(_Scene), dp, ctypes.c_double, ctypes.c_int,
                                                     dp, ctypes.c_int, dp, ctypes.c_uint64, ctypes.c_uint32,
                                                     ctypes.c_uint32]
            L.oracle_neumann_data_sample.restype = ctypes.c_double
            L.oracle_bessel_k0.argtypes = [ctypes.c_double]
            L.oracle_bessel_k0.restype = ctypes.c_double
            L.oracle_gradient_factor.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
            L.oracle_gradient_factor.restype = ctypes.c_double
            L.oracle_closest_point.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, dp, dp, dp,
                                               ip, dp]
            L.oracle_closest_point.restype = ctypes.c_int
            L.oracle_run_walks.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, dp, ctypes.c_int,
                                           ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(_WalkOut)]
            L.oracle_run_walks.restype = ctypes.c_int
            L.oracle_inside.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, dp, ip]
            L.oracle_inside.restype = ctypes.c_int
            L.oracle_num_threads.argtypes = []
            L.oracle_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if a is not None else None


@dataclass
class Problem:
    """A Dirichlet screened-Poisson problem on a polyline / triangle-mesh boundary.

    data_kind 'mapped': per-vertex data g_vert (and optional dg_vert, n_vert x N)
    data_kind 'field' : g = c0 + c.x + x^T A x with field = [c0, c(3), Axx, Ayy, Azz, Axy, Axz, Ayz]
    f is the constant source of  -Lap u + sigma u = f  (the sign Algorithm 1 uses).
    """
    vert: np.ndarray
    elem: np.ndarray
    jac: Optional[np.ndarray] = None
    data_kind: str = "mapped"
    g_vert: Optional[np.ndarray] = None
    dg_vert: Optional[np.ndarray] = None
    field: Optional[np.ndarray] = None
    sigma: float = 0.0
    f: float = 0.0
    eps: float = 1e-3
    h: float = 1e-2
    K: int = 1
    max_steps: int = 1 << 14
    seed: int = 0x12964
    cv_elem: Optional[np.ndarray] = None      # (n_elem, 4): q, t of the nested walks' surrogate grad u = q n + t
    dudn_mode: int = 0                        # 0: backward difference (Eq. dudn_fd_estimate), 1: ball gradient
    neumann: Optional[np.ndarray] = None      # (n_elem,) flags: 1 for elements of the reflecting Neumann part
    neumann_h: Optional[np.ndarray] = None    # (n_elem,) Neumann data du/dn (out of the domain); None: zero
    _keep: list = dc_field(default_factory=list, repr=False)

    @property
    def dim(self) -> int:
        return int(self.vert.shape[1])

    @property
    def n_param(self) -> int:
        return 0 if self.jac is None else int(self.jac.shape[2])

    def _struct(self) -> _Scene:
        v = np.ascontiguousarray(self.vert, dtype=np.float64)
        e = np.ascontiguousarray(self.elem, dtype=np.int32)
        jac = None if self.jac is None else np.ascontiguousarray(self.jac, dtype=np.float64)
        g = None if self.g_vert is None else np.ascontiguousarray(self.g_vert, dtype=np.float64)
        dg = None if self.dg_vert is None else np.ascontiguousarray(self.dg_vert, dtype=np.float64)
        cq = None if self.cv_elem is None else np.ascontiguousarray(self.cv_elem, dtype=np.float64).reshape(-1, 4)
        nm = None if self.neumann is None else np.ascontiguousarray(self.neumann, dtype=np.int32)
        nh = None if self.neumann_h is None else np.ascontiguousarray(self.neumann_h, dtype=np.float64)
        self._keep = [v, e, jac, g, dg, cq, nm, nh]
        s = _Scene()
        s.dim = v.shape[1]
        s.n_vert = v.shape[0]
        s.vert = _dp(v)
        s.n_elem = e.shape[0]
        s.elem = _ip(e)
        s.n_param = 0 if jac is None else jac.shape[2]
        s.jac = _dp(jac)
        s.data_kind = 1 if self.data_kind == "field" else 0
        if self.data_kind == "mapped" and g is None:
            raise ValueError("mapped data needs g_vert")
        s.g_vert = _dp(g)
        s.dg_vert = _dp(dg)
        s.field_kind = 0
        fv = np.zeros(10) if self.field is None else np.asarray(self.field, dtype=np.float64)
        for i in range(10):
            s.field[i] = float(fv[i]) if i < len(fv) else 0.0
        s.sigma = float(self.sigma)
        s.f = float(self.f)
        s.eps = float(self.eps)
        s.h = float(self.h)
        s.K = int(self.K)
        s.max_steps = int(self.max_steps)
        s.seed_lo = self.seed & 0xFFFFFFFF
        s.seed_hi = (self.seed >> 32) & 0xFFFFFFFF
        s.cv_elem = _dp(cq)
        s.dudn_mode = int(self.dudn_mode)
        s.neumann = _ip(nm)
        s.neumann_h = _dp(nh)
        return s


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, out)
    return np.array(list(out), dtype=np.uint32)


def uniform(x: int) -> float:
    return lib().oracle_uniform(int(x) & 0xFFFFFFFF)


def alpha(dim: int, sigma: float, d: float) -> float:
    return lib().oracle_alpha(dim, sigma, d)


def source_weight(dim: int, sigma: float, d: float, rho: float) -> float:
    """|B(d)| * G_d(rho d): Algorithm 1's source weight per unit source."""
    return lib().oracle_source_weight(dim, sigma, d, rho)


def ray_neumann(prob: "Problem", x, v, tmax: float, skip: int = -1, n_skip=None, skip2: int = -1, n_skip2=None):
    """First crossing of the ray x + t v (t <= tmax, plus the walk's slack) with
    the Neumann part, for a walk sitting on element `skip` (and `skip2` at an
    edge) with outward normals n_skip (n_skip2).  Returns (t, element or -1)."""
    s = prob._struct()
    d = prob.dim
    xx = np.zeros(3); xx[:d] = np.asarray(x, dtype=np.float64)[:d]
    vv = np.zeros(3); vv[:d] = np.asarray(v, dtype=np.float64)[:d]
    a = None if n_skip is None else np.ascontiguousarray(np.resize(np.asarray(n_skip, dtype=np.float64), 3))
    b = None if n_skip2 is None else np.ascontiguousarray(np.resize(np.asarray(n_skip2, dtype=np.float64), 3))
    if a is not None and d == 2: a[2] = 0.0
    if b is not None and d == 2: b[2] = 0.0
    e = ctypes.c_int(-1)
    t = lib().oracle_ray_neumann(ctypes.byref(s), _dp(xx), _dp(vv), float(tmax), int(skip), _dp(a), int(skip2),
                                 _dp(b), ctypes.byref(e))
    return float(t), int(e.value)


def neumann_data_sample(prob: "Problem", x, R: float, on: int = -1, n_on=None, on2: int = -1, n2=None,
                        walk_id: int = 0, step: int = 0, phase: int = 0) -> float:
    """The Neumann-data term of one walk-on-stars step from x with star radius
    R, for a walk on element `on` (and `on2` at an edge; -1: none) with outward
    normals n_on (n2), drawn at step `step` of phase `phase` of walk walk_id."""
    s = prob._struct()
    d = prob.dim
    xx = np.zeros(3); xx[:d] = np.asarray(x, dtype=np.float64)[:d]
    a = None if n_on is None else np.ascontiguousarray(np.resize(np.asarray(n_on, dtype=np.float64), 3))
    b = None if n2 is None else np.ascontiguousarray(np.resize(np.asarray(n2, dtype=np.float64), 3))
    if a is not None and d == 2: a[2] = 0.0
    if b is not None and d == 2: b[2] = 0.0
    return float(lib().oracle_neumann_data_sample(ctypes.byref(s), _dp(xx), float(R), int(on), _dp(a), int(on2),
                                                  _dp(b), int(walk_id), int(step), int(phase)))


def turn_inward(v: np.ndarray, n_on, n2=None) -> np.ndarray:
    """Directions drawn on the Neumann part turned into the domain: v (n x 3)
    for a walk on a side with outward normal n_on, or on the edge of two sides
    (outward normals n_on, n2)."""
    v = np.array(v, dtype=np.float64, order="C").reshape(-1, 3)
    a = np.ascontiguousarray(n_on, dtype=np.float64).reshape(3)
    b = None if n2 is None else np.ascontiguousarray(n2, dtype=np.float64).reshape(3)
    lib().oracle_turn_inward(v.shape[0], _dp(v), _dp(a), _dp(b))
    return v


def star_weight(dim: int, sigma: float, t: float, R: float) -> float:
    """Survival weight of a walk-on-stars step of length t in the ball of radius R."""
    return lib().oracle_star_weight(dim, sigma, t, R)


def bessel_k0(x: float) -> float:
    """K0(x) from std::cyl_bessel_k (the library routine the source weight uses)."""
    return lib().oracle_bessel_k0(float(x))


def gradient_factor(dim: int, sigma: float, R: float) -> float:
    """F with grad u(c) = F E[n_y u(y)] over the sphere of radius R about c."""
    return lib().oracle_gradient_factor(dim, sigma, R)


def closest_point(prob: Problem, pts: np.ndarray):
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, prob.dim)
    n = pts.shape[0]
    dist = np.zeros(n)
    xbar = np.zeros((n, prob.dim))
    elem = np.zeros(n, dtype=np.int32)
    bary = np.zeros((n, 2))
    s = prob._struct()
    lib().oracle_closest_point(ctypes.byref(s), n, _dp(pts), _dp(dist), _dp(xbar), _ip(elem), _dp(bary))
    return dist, xbar, elem, bary


def inside(prob: Problem, pts: np.ndarray) -> np.ndarray:
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, prob.dim)
    out = np.zeros(pts.shape[0], dtype=np.int32)
    s = prob._struct()
    lib().oracle_inside(ctypes.byref(s), pts.shape[0], _dp(pts), _ip(out))
    return out.astype(bool)


def run_walks(prob: Problem, xq: np.ndarray, walks_per_point: int, differential: bool = False,
              walk_id_base: int = 0, threads: int = 0) -> dict:
    """Run walks_per_point walks from every query point.

    Walk (p, w) uses Philox walk id walk_id_base + p * W + w; every output is
    indexed by p * W + w.  Returns u_hat, x1 (the main walk's point after its
    first sphere step, NaN if it never moved), x_end (where the main walk
    stopped) and, for differential walks, udot
    (n x N), dudn, u_off, u_plain, disp_n, disp_t (the nested walks' mean
    estimate without the control variate and their mean normal / tangential
    displacements), elem, bary, normal, xbar, kind and steps
    ((K + 1) slots: the main walk, then the nested walks).
    """
    xq = np.ascontiguousarray(xq, dtype=np.float64).reshape(-1, prob.dim)
    n = xq.shape[0] * walks_per_point
    K1 = prob.K + 1
    P = prob.n_param
    out = {
        "u_hat": np.zeros(n),
        "elem": np.zeros(n, dtype=np.int32),
        "bary": np.zeros((n, 2)),
        "xbar": np.zeros((n, 3)),
        "kind": np.zeros((n, K1), dtype=np.int32),
        "steps": np.zeros((n, K1), dtype=np.int32),
        "x1": np.zeros((n, 3)),
        "x_end": np.zeros((n, 3)),
    }
    if differential:
        out["udot"] = np.zeros((n, P))
        out["dudn"] = np.zeros(n)
        out["u_off"] = np.zeros(n)
        out["normal"] = np.zeros((n, 3))
        out["u_plain"] = np.zeros(n)
        out["disp_n"] = np.zeros(n)
        out["disp_t"] = np.zeros(n)
    o = _WalkOut()
    o.u_hat = _dp(out["u_hat"])
    o.udot = _dp(out.get("udot")) if P > 0 and differential else None
    o.dudn = _dp(out.get("dudn"))
    o.u_off = _dp(out.get("u_off"))
    o.elem = _ip(out["elem"])
    o.bary = _dp(out["bary"])
    o.normal = _dp(out.get("normal"))
    o.xbar = _dp(out["xbar"])
    o.kind = _ip(out["kind"])
    o.steps = _ip(out["steps"])
    o.x1 = _dp(out["x1"])
    o.x_end = _dp(out["x_end"])
    o.u_plain = _dp(out.get("u_plain"))
    o.disp_n = _dp(out.get("disp_n"))
    o.disp_t = _dp(out.get("disp_t"))
    s = prob._struct()
    rc = lib().oracle_run_walks(ctypes.byref(s), xq.shape[0], _dp(xq), walks_per_point,
                                walk_id_base, 1 if differential else 0, threads, ctypes.byref(o))
    if rc != 0:
        raise ValueError("oracle_run_walks rejected its arguments")
    if not differential:
        out["kind"] = out["kind"][:, :1]
        out["steps"] = out["steps"][:, :1]
    return out


def num_threads() -> int:
    return lib().oracle_num_threads()
