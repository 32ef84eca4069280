"""FP64 CPU oracle (test infrastructure only).

A plain, slow restatement of the randomized pose search and TSDF fusion of
PROFusion (arXiv 2509.24236, Sec. III and III-B, defaults of Sec. IV-A) in C,
compiled with gcc and called through ctypes.  Only the tests, the smoke check
and the bench's CPU-baseline leg may use it; the CUDA library never does, and
the two share no code.

Parity pins for every function live in tests/test_oracle_pins.py and (the
alignment loss, its derivatives and the polish) tests/test_oracle_align.py;
the oracle is pinned by closed forms, invariants and FP64 finite
differences, never by the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

MAX_ITERS = 32


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, FP64, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Intr(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("depth_min", C.c_double), ("depth_max", C.c_double)]


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("voxel_size", C.c_double),
                ("trunc", C.c_double), ("origin", C.c_double * 3), ("max_weight", C.c_int)]


class _Params(C.Structure):
    _fields_ = [("n_iters", C.c_int), ("k_sched", C.c_int * 3), ("decim_sched", C.c_int * 3),
                ("s0_deg", C.c_double), ("s0_cm", C.c_double), ("beta", C.c_double),
                ("update_mode", C.c_int), ("compose_mode", C.c_int), ("min_valid_frac", C.c_double)]


class _Stats(C.Structure):
    M = MAX_ITERS
    _fields_ = [("n_points", C.c_int), ("n_iters", C.c_int), ("lost", C.c_int), ("pad", C.c_int),
                ("E0", C.c_double * M), ("E_best", C.c_double * M), ("E_new", C.c_double * M),
                ("best", C.c_int * M), ("n_adv", C.c_int * M), ("n_valid0", C.c_int * M),
                ("n_eval", C.c_int * M), ("k_used", C.c_int * M), ("pad2", C.c_int),
                ("s", (C.c_double * 2) * M), ("pose", (C.c_double * 12) * M),
                ("adv_margin", C.c_double * M), ("best_gap", C.c_double * M)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        dp, fp, lp = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_long)
        lib.or_backproject.restype = C.c_long
        lib.or_backproject.argtypes = [fp, C.POINTER(_Intr), C.c_int, dp]
        lib.or_sample.restype = C.c_int
        lib.or_sample.argtypes = [dp, dp, C.POINTER(_Grid), dp, dp]
        lib.or_fitness.restype = None
        lib.or_fitness.argtypes = [dp, dp, C.POINTER(_Grid), dp, C.c_long, C.c_long, dp, C.c_int,
                                   dp, lp, dp, lp, C.c_double, dp, C.c_int]
        lib.or_sample_band.restype = C.c_int
        lib.or_sample_band.argtypes = [dp, dp, C.POINTER(_Grid), dp, dp]
        lib.or_so3_exp.restype = None
        lib.or_so3_exp.argtypes = [dp, dp]
        lib.or_particles.restype = None
        lib.or_particles.argtypes = [fp, C.c_int, dp, C.c_double, C.c_double, C.c_int, dp]
        lib.or_track.restype = C.c_int
        lib.or_track.argtypes = [dp, dp, C.POINTER(_Grid), fp, C.POINTER(_Intr), C.POINTER(_Params),
                                 fp, C.c_int, dp, dp, C.POINTER(_Stats)]
        lib.or_integrate.restype = C.c_long
        lib.or_integrate.argtypes = [dp, dp, C.POINTER(_Grid), fp, C.POINTER(_Intr), dp,
                                     C.POINTER(C.c_ubyte), C.c_double, C.c_double]
        lib.or_raycast.restype = None
        lib.or_raycast.argtypes = [dp, dp, C.POINTER(_Grid), C.POINTER(_Intr), dp, C.c_double, dp, dp]
        lib.or_perturb_pose.restype = None
        lib.or_perturb_pose.argtypes = [dp, dp, dp]
        lib.or_align_loss.restype = None
        lib.or_align_loss.argtypes = [dp, dp, C.POINTER(_Grid), dp, C.c_long, dp, dp, dp, lp, dp, dp]
        lib.or_polish.restype = C.c_int
        lib.or_polish.argtypes = [dp, dp, C.POINTER(_Grid), dp, C.c_long, dp, C.c_int, dp]
        lib.or_num_threads.restype = C.c_int
        _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _intr(intr) -> _Intr:
    return _Intr(intr.width, intr.height, intr.fx, intr.fy, intr.cx, intr.cy, intr.depth_min, intr.depth_max)


def _grid(g, max_weight: int = 255) -> _Grid:
    return _Grid(g.nx, g.ny, g.nz, g.voxel_size, g.trunc, (C.c_double * 3)(*g.origin), max_weight)


def _pose12(P) -> np.ndarray:
    P = np.asarray(P, dtype=np.float64)
    return _f64(P[:3, :4].reshape(12) if P.shape in ((4, 4), (3, 4)) else P.reshape(12))


def num_threads() -> int:
    return int(_load().or_num_threads())


# ---------------------------------------------------------------------------
class Volume:
    """FP64 TSDF grid (normalised tsdf, weights), x-fastest node order."""

    def __init__(self, grid, tsdf=None, weight=None, max_weight: int = 255):
        self.grid = grid
        self.max_weight = max_weight
        n = grid.n_nodes
        self.tsdf = _f64(np.ones(n) if tsdf is None else tsdf)
        self.weight = _f64(np.zeros(n) if weight is None else weight)

    def _g(self):
        return _grid(self.grid, self.max_weight)


def backproject(depth, intr, stride: int = 1) -> np.ndarray:
    d = _f32(depth)
    out = np.empty((max(1, d.size), 3), dtype=np.float64)
    n = _load().or_backproject(_p(d, C.c_float), C.byref(_intr(intr)), int(stride), _p(out, C.c_double))
    return out[:n].copy()


def sample(vol: Volume, q, band: bool = False) -> float | None:
    """Trilinear TSDF at q; None unless the cell is inside the grid with all
    eight nodes observed (and, with band=True, all within the truncation)."""
    qq = _f64(q)
    v = C.c_double()
    fn = _load().or_sample_band if band else _load().or_sample
    ok = fn(_p(vol.tsdf, C.c_double), _p(vol.weight, C.c_double), C.byref(vol._g()),
            _p(qq, C.c_double), C.byref(v))
    return v.value if ok else None


@dataclass
class FitnessResult:
    S: np.ndarray
    C: np.ndarray
    E: np.ndarray
    amb: np.ndarray | None = None    # ambiguous points per pose (excluded from S, C)
    vals: np.ndarray | None = None   # their values when counted, K x cap


def fitness(vol: Volume, points, poses, stride: int = 1, ambiguity: bool = False,
            eps_g: float = 1e-4, cap: int = 32) -> FitnessResult:
    """E_k for K row-major 3x4 poses (K x 12) against points (N x 3).

    With ambiguity=True, points within eps_g voxels of a cell face across
    which validity changes are left out of S, C, E and reported instead
    (count per pose in `amb`, their values in `vals`)."""
    pts = _f64(np.asarray(points)[:, :3])
    T = _f64(np.asarray(poses).reshape(-1, 12))
    K = T.shape[0]
    S = np.empty(K)
    Cn = np.empty(K, dtype=np.int64)
    E = np.empty(K)
    A = np.empty(K, dtype=np.int64) if ambiguity else None
    V = np.zeros((K, cap)) if ambiguity else None
    _load().or_fitness(_p(vol.tsdf, C.c_double), _p(vol.weight, C.c_double), C.byref(vol._g()),
                       _p(pts, C.c_double), pts.shape[0], int(stride), _p(T, C.c_double), K,
                       _p(S, C.c_double), _p(Cn, C.c_long), _p(E, C.c_double),
                       _p(A, C.c_long) if A is not None else None, eps_g,
                       _p(V, C.c_double) if V is not None else None, cap)
    return FitnessResult(S, Cn, E, A, V)


def so3_exp(w) -> np.ndarray:
    ww = _f64(w)
    R = np.empty(9)
    _load().or_so3_exp(_p(ww, C.c_double), _p(R, C.c_double))
    return R.reshape(3, 3)


def particles(templ, K: int, P, s_deg: float, s_cm: float, compose_mode: int = 0) -> np.ndarray:
    t = _f32(templ)
    out = np.empty((K, 12))
    _load().or_particles(_p(t, C.c_float), int(K), _p(_pose12(P), C.c_double), s_deg, s_cm,
                         int(compose_mode), _p(out, C.c_double))
    return out


@dataclass
class TrackParams:
    n_iters: int = 20
    k_sched: tuple = (1024, 3072, 10240)
    decim_sched: tuple = (8, 16, 32)
    s0_deg: float = 10.0
    s0_cm: float = 10.0
    beta: float = 0.1
    update_mode: int = 0
    compose_mode: int = 0
    min_valid_frac: float = 0.0


@dataclass
class TrackResult:
    pose: np.ndarray       # 4x4
    lost: bool
    stats: dict


def track(vol: Volume, depth, intr, templ, P0, params: TrackParams) -> TrackResult:
    t = _f32(templ)
    d = _f32(depth)
    prm = _Params(params.n_iters, (C.c_int * 3)(*params.k_sched), (C.c_int * 3)(*params.decim_sched),
                  params.s0_deg, params.s0_cm, params.beta, params.update_mode, params.compose_mode,
                  params.min_valid_frac)
    out = np.empty(12)
    st = _Stats()
    lost = _load().or_track(_p(vol.tsdf, C.c_double), _p(vol.weight, C.c_double), C.byref(vol._g()),
                            _p(d, C.c_float), C.byref(_intr(intr)), C.byref(prm), _p(t, C.c_float),
                            t.shape[0], _p(_pose12(P0), C.c_double), _p(out, C.c_double), C.byref(st))
    n = st.n_iters
    stats = {
        "n_points": st.n_points, "n_iters": n,
        "E0": np.array(st.E0[:n]), "E_best": np.array(st.E_best[:n]), "E_new": np.array(st.E_new[:n]),
        "best": np.array(st.best[:n]), "n_adv": np.array(st.n_adv[:n]),
        "n_valid0": np.array(st.n_valid0[:n]), "n_eval": np.array(st.n_eval[:n]),
        "k_used": np.array(st.k_used[:n]),
        "s": np.array([[st.s[i][0], st.s[i][1]] for i in range(n)]),
        "pose": np.array([list(st.pose[i]) for i in range(n)]),
        "adv_margin": np.array(st.adv_margin[:n]), "best_gap": np.array(st.best_gap[:n]),
    }
    P = np.eye(4)
    P[:3, :4] = out.reshape(3, 4)
    return TrackResult(P, bool(lost), stats)


def integrate(vol: Volume, depth, intr, pose, ambiguity: bool = False,
              eps_px: float = 1e-3, eps_m: float = 1e-6):
    """Fuse one depth image in place.  Returns the ambiguity mask if asked."""
    d = _f32(depth)
    mask = np.zeros(vol.grid.n_nodes, dtype=np.uint8) if ambiguity else None
    _load().or_integrate(_p(vol.tsdf, C.c_double), _p(vol.weight, C.c_double), C.byref(vol._g()),
                         _p(d, C.c_float), C.byref(_intr(intr)), _p(_pose12(pose), C.c_double),
                         _p(mask, C.c_ubyte) if mask is not None else None, eps_px, eps_m)
    return mask


def raycast(vol: Volume, intr, pose, step: float | None = None):
    """(depth H x W, normals H x W x 3) of the fused surface."""
    step = 0.5 * vol.grid.trunc if step is None else step
    depth = np.empty((intr.height, intr.width))
    normals = np.empty((intr.height, intr.width, 3))
    _load().or_raycast(_p(vol.tsdf, C.c_double), _p(vol.weight, C.c_double), C.byref(vol._g()),
                       C.byref(_intr(intr)), _p(_pose12(pose), C.c_double), float(step),
                       _p(depth, C.c_double), _p(normals, C.c_double))
    return depth, normals


# ---------------------------------------------------------------------------
# Alignment loss, its derivatives and the Gauss-Newton polish
# ---------------------------------------------------------------------------

def perturb_pose(P, xi) -> np.ndarray:
    """4x4 pose of q = Exp(omega) (R x + t) + v, xi = (omega, v)."""
    out = np.empty(12)
    _load().or_perturb_pose(_p(_pose12(P), C.c_double), _p(_f64(xi), C.c_double), _p(out, C.c_double))
    T = np.eye(4)
    T[:3, :4] = out.reshape(3, 4)
    return T


@dataclass
class AlignResult:
    loss: float            # sum of tsdf^2 over the valid points
    count: int             # valid points
    grad_xi: np.ndarray    # dL/dxi at xi (6)
    grad_tsdf: np.ndarray | None  # dL/dV per node, or None


def align_loss(vol: Volume, points, pose, xi=None, grad_tsdf: bool = False) -> AlignResult:
    pts = _f64(np.asarray(points)[:, :3])
    gV = np.zeros(vol.grid.n_nodes) if grad_tsdf else None
    L = C.c_double()
    Cn = C.c_long()
    g = np.empty(6)
    _load().or_align_loss(_p(vol.tsdf, C.c_double), _p(vol.weight, C.c_double), C.byref(vol._g()),
                          _p(pts, C.c_double), pts.shape[0], _p(_pose12(pose), C.c_double),
                          _p(_f64(xi), C.c_double) if xi is not None else None, C.byref(L), C.byref(Cn),
                          _p(g, C.c_double), _p(gV, C.c_double) if gV is not None else None)
    return AlignResult(L.value, Cn.value, g, gV)


def polish(vol: Volume, points, pose, steps: int = 10):
    """(pose 4x4 after `steps` damped Gauss-Newton candidates, accepted
    steps, objective trace of steps + 1 values)."""
    pts = _f64(np.asarray(points)[:, :3])
    T = _pose12(pose).copy()
    trace = np.empty(steps + 1)
    acc = _load().or_polish(_p(vol.tsdf, C.c_double), _p(vol.weight, C.c_double), C.byref(vol._g()),
                            _p(pts, C.c_double), pts.shape[0], _p(T, C.c_double), int(steps),
                            _p(trace, C.c_double))
    P = np.eye(4)
    P[:3, :4] = T.reshape(3, 4)
    return P, int(acc), trace
