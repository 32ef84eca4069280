"""Thin ctypes binding of libprofusion (include/profusion.h).

The functions named pf_* mirror the C ABI one to one: they only marshal
arguments (torch CUDA tensors -> device pointers, the current torch stream ->
cudaStream_t) and return the pf_status.  `Volume` wraps them for convenience.
Every computation happens in the CUDA kernels of libprofusion; there is no
other code path, and importing the binding fails loudly when the library has
not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libprofusion.so")

PF_OK, PF_ERR_INVALID_ARG, PF_ERR_OOM, PF_ERR_CUDA, PF_ERR_TIMEOUT, PF_ERR_TRACK_LOST, PF_ERR_UNSUPPORTED = range(7)
PF_F32, PF_F16, PF_BF16, PF_FP8E4M3 = range(4)
PF_MAX_ITERS = 32


class pf_intrinsics(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("depth_min", C.c_float), ("depth_max", C.c_float)]


class pf_volume_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("voxel_size", C.c_float),
                ("trunc", C.c_float), ("origin", C.c_float * 3), ("tsdf_dtype", C.c_int),
                ("weight_u8", C.c_int), ("max_weight", C.c_int), ("cell_view", C.c_int),
                ("search_dtype", C.c_int)]


class pf_track_params(C.Structure):
    _fields_ = [("n_iters", C.c_int), ("k_sched", C.c_int * 3), ("decim_sched", C.c_int * 3),
                ("init_rot_deg", C.c_double), ("init_trans_cm", C.c_double), ("beta", C.c_double),
                ("templates_dev", C.c_void_p), ("k_max", C.c_int), ("update_mode", C.c_int),
                ("compose_mode", C.c_int), ("min_valid_frac", C.c_float)]


class pf_track_stats(C.Structure):
    M = PF_MAX_ITERS
    _fields_ = [("n_points", C.c_int), ("n_iters", C.c_int), ("status", C.c_int), ("reserved", C.c_int),
                ("E0", C.c_float * M), ("E_best", C.c_float * M), ("E_new", C.c_float * M),
                ("best", C.c_int * M), ("n_adv", C.c_int * M), ("n_valid0", C.c_int * M),
                ("n_eval", C.c_int * M), ("k_used", C.c_int * M),
                ("s", (C.c_double * 2) * M), ("pose", (C.c_double * 12) * M)]

    def to_dict(self) -> dict:
        n = self.n_iters
        return {
            "n_points": self.n_points, "n_iters": n, "status": self.status,
            "E0": np.array(self.E0[:n], dtype=np.float32), "E_best": np.array(self.E_best[:n], dtype=np.float32),
            "E_new": np.array(self.E_new[:n], dtype=np.float32), "best": np.array(self.best[:n]),
            "n_adv": np.array(self.n_adv[:n]), "n_valid0": np.array(self.n_valid0[:n]),
            "n_eval": np.array(self.n_eval[:n]), "k_used": np.array(self.k_used[:n]),
            "s": np.array([[self.s[i][0], self.s[i][1]] for i in range(n)]),
            "pose": np.array([list(self.pose[i]) for i in range(n)]),
        }


EXPORTS = ["pf_create_volume", "pf_destroy_volume", "pf_reset_volume", "pf_volume_upload", "pf_volume_download",
           "pf_integrate", "pf_integrate_async", "pf_pose_compose", "pf_backproject", "pf_fitness", "pf_fitness_noalloc", "pf_track_frame", "pf_track_frame_async",
           "pf_track_reserve", "pf_raycast", "pf_set_fitness_variant", "pf_status_string", "pf_launch_count",
           "pf_set_kernel_timing", "pf_kernel_timing", "pf_align_loss", "pf_polish",
           "pf_batch_create", "pf_batch_destroy", "pf_batch_buffers", "pf_batch_fuse", "pf_batch_step",
           "pf_batch_autotune", "pf_batch_set_points_per_block", "pf_volume_info", "pf_alloc_count", "pf_volume_last_error", "pf_batch_set_mapping_threshold",
           "pf_batch_tuning",
           "pf_gather_probe"]

_lib = None


class ProfusionError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libprofusion.so (built in-tree by build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libprofusion.so is not built ({path}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` -- there is no fallback path")
    lib = C.CDLL(path)
    vp, ip, dp, fp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_float)
    st = C.c_int
    sig = {
        "pf_create_volume": (st, [C.POINTER(pf_volume_desc), vp, C.POINTER(vp)]),
        "pf_destroy_volume": (st, [vp]),
        "pf_reset_volume": (st, [vp, vp]),
        "pf_volume_upload": (st, [vp, fp, fp]),
        "pf_volume_download": (st, [vp, fp, fp]),
        "pf_integrate": (st, [vp, vp, C.POINTER(pf_intrinsics), dp, vp]),
        "pf_integrate_async": (st, [vp, vp, C.POINTER(pf_intrinsics), vp, vp]),
        "pf_pose_compose": (st, [vp, vp, vp, vp]),
        "pf_backproject": (st, [vp, C.POINTER(pf_intrinsics), vp, C.c_int, vp, vp]),
        "pf_fitness": (st, [vp, vp, C.c_int, vp, C.c_int, vp, vp, vp]),
        "pf_fitness_noalloc": (st, [vp, vp, C.c_int, vp, C.c_int, vp, vp, vp]),
        "pf_track_frame": (st, [vp, vp, C.POINTER(pf_intrinsics), C.POINTER(pf_track_params), dp, dp,
                                C.POINTER(pf_track_stats), vp]),
        "pf_track_frame_async": (st, [vp, vp, C.POINTER(pf_intrinsics), C.POINTER(pf_track_params), vp, vp,
                                      vp, vp]),
        "pf_track_reserve": (st, [vp, C.c_int, C.c_int]),
        "pf_raycast": (st, [vp, C.POINTER(pf_intrinsics), dp, vp, vp, vp]),
        "pf_set_fitness_variant": (st, [vp, C.c_int]),
        "pf_volume_info": (st, [vp, C.POINTER(C.c_ulonglong), C.POINTER(C.c_int)]),
        "pf_status_string": (C.c_char_p, [st]),
        "pf_launch_count": (C.c_ulonglong, []),
        "pf_alloc_count": (C.c_ulonglong, []),
        "pf_volume_last_error": (st, [vp, C.c_int]),
        "pf_gather_probe": (st, [vp, C.c_longlong, C.c_int, C.c_int, vp, C.POINTER(C.c_longlong), vp]),
        "pf_set_kernel_timing": (st, [C.c_int]),
        "pf_kernel_timing": (st, [C.c_char_p, dp, C.POINTER(C.c_longlong)]),
        "pf_align_loss": (st, [vp, vp, vp, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp]),
        "pf_polish": (st, [vp, vp, vp, C.c_int, vp, C.c_int, vp, vp, vp]),
        "pf_batch_create": (st, [C.c_int, C.POINTER(vp), C.POINTER(pf_intrinsics), C.POINTER(pf_track_params),
                                 C.c_int, C.POINTER(vp)]),
        "pf_batch_destroy": (st, [vp]),
        "pf_batch_buffers": (st, [vp, C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]),
        "pf_batch_fuse": (st, [vp, vp]),
        "pf_batch_step": (st, [vp, vp]),
        "pf_batch_autotune": (st, [vp, vp, C.POINTER(C.c_int)]),
        "pf_batch_set_points_per_block": (st, [vp, C.c_int]),
        "pf_batch_set_mapping_threshold": (st, [vp, C.c_float]),
        "pf_batch_tuning": (st, [vp, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().pf_status_string(status).decode()


def _check(status: int, what: str, ok=(PF_OK,)):
    if status not in ok:
        raise ProfusionError(status, what)
    return status


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def intrinsics(intr) -> pf_intrinsics:
    """pf_intrinsics from any object with width/height/fx/fy/cx/cy/depth_min/depth_max."""
    return pf_intrinsics(intr.width, intr.height, intr.fx, intr.fy, intr.cx, intr.cy,
                         getattr(intr, "depth_min", 0.1), getattr(intr, "depth_max", 8.0))


def _pose16(P) -> C.Array:
    """double[16] row-major 4x4 from a 4x4, 3x4 or flat 12/16 pose."""
    P = np.asarray(P, dtype=np.float64).reshape(-1, 4)
    if P.shape[0] not in (3, 4):
        raise ValueError("pose must be 3x4 or 4x4")
    full = np.eye(4)
    full[:3] = P[:3]
    return (C.c_double * 16)(*full.reshape(16))


# ---------------------------------------------------------------------------
# C-ABI mirrors (same names, argument marshalling only)
# ---------------------------------------------------------------------------

def pf_create_volume(desc: pf_volume_desc, stream=None) -> C.c_void_p:
    out = C.c_void_p()
    _check(load().pf_create_volume(C.byref(desc), _stream(stream), C.byref(out)), "pf_create_volume")
    return out


def pf_destroy_volume(vol) -> int:
    return load().pf_destroy_volume(vol)


def pf_reset_volume(vol, stream=None) -> int:
    return _check(load().pf_reset_volume(vol, _stream(stream)), "pf_reset_volume")


def pf_volume_upload(vol, tsdf: np.ndarray, weight: np.ndarray) -> int:
    t = np.ascontiguousarray(tsdf, dtype=np.float32)
    w = np.ascontiguousarray(weight, dtype=np.float32)
    return _check(load().pf_volume_upload(vol, t.ctypes.data_as(C.POINTER(C.c_float)),
                                          w.ctypes.data_as(C.POINTER(C.c_float))), "pf_volume_upload")


def pf_volume_download(vol, n_nodes: int):
    t = np.empty(n_nodes, dtype=np.float32)
    w = np.empty(n_nodes, dtype=np.float32)
    _check(load().pf_volume_download(vol, t.ctypes.data_as(C.POINTER(C.c_float)),
                                     w.ctypes.data_as(C.POINTER(C.c_float))), "pf_volume_download")
    return t, w


def pf_integrate(vol, depth, intr, pose, stream=None) -> int:
    import torch
    return _check(load().pf_integrate(vol, _dptr(depth, torch.float32), C.byref(intrinsics(intr)),
                                      _pose16(pose), _stream(stream)), "pf_integrate")


def pf_integrate_async(vol, depth, intr, pose_dev, stream=None) -> int:
    import torch
    return _check(load().pf_integrate_async(vol, _dptr(depth, torch.float32), C.byref(intrinsics(intr)),
                                            _dptr(pose_dev, torch.float64), _stream(stream)), "pf_integrate_async")


def pf_pose_compose(a_dev, b_dev, out_dev, stream=None) -> int:
    import torch
    return _check(load().pf_pose_compose(_dptr(a_dev, torch.float64), _dptr(b_dev, torch.float64),
                                         _dptr(out_dev, torch.float64), _stream(stream)), "pf_pose_compose")


def pf_backproject(depth, intr, points, n_out, stream=None) -> int:
    import torch
    return _check(load().pf_backproject(_dptr(depth, torch.float32), C.byref(intrinsics(intr)),
                                        _dptr(points, torch.float32), points.numel() // 4,
                                        _dptr(n_out, torch.int32), _stream(stream)), "pf_backproject")


def pf_fitness(vol, points, n: int, poses, k: int, fitness, count, stream=None) -> int:
    import torch
    return _check(load().pf_fitness(vol, _dptr(points, torch.float32) if n > 0 else None, n,
                                    _dptr(poses, torch.float32), k, _dptr(fitness, torch.float32),
                                    _dptr(count, torch.int32), _stream(stream)), "pf_fitness")


def pf_align_loss(vol, points, counts, n_max: int, n_frames: int, poses, xi, dloss, loss, count, grad_xi,
                  grad_tsdf, stream=None) -> int:
    import torch
    return _check(load().pf_align_loss(vol, _dptr(points, torch.float32) if n_max > 0 else None,
                                       _dptr(counts, torch.int32), n_max, n_frames, _dptr(poses, torch.float64),
                                       _dptr(xi, torch.float64), _dptr(dloss, torch.float64),
                                       _dptr(loss, torch.float64), _dptr(count, torch.int32),
                                       _dptr(grad_xi, torch.float64), _dptr(grad_tsdf, torch.float32),
                                       _stream(stream)), "pf_align_loss")


def pf_polish(vol, points, n_dev, n_max: int, pose, steps: int, trace=None, accepted=None, stream=None) -> int:
    import torch
    return _check(load().pf_polish(vol, _dptr(points, torch.float32) if n_max > 0 else None,
                                   _dptr(n_dev, torch.int32), n_max, _dptr(pose, torch.float64), int(steps),
                                   _dptr(trace, torch.float64), _dptr(accepted, torch.int32), _stream(stream)),
                  "pf_polish")


PF_NOALLOC_MAX_SLOTS = 65536


def pf_fitness_noalloc(vol, points, n: int, poses, k: int, fitness, count, stream=None) -> int:
    """pf_fitness without any device allocation (fixed scratch inside the
    library; calls must not overlap on the GPU).  Returns the pf_status."""
    import torch
    return load().pf_fitness_noalloc(vol, _dptr(points, torch.float32) if n > 0 else None, n,
                                     _dptr(poses, torch.float32), k, _dptr(fitness, torch.float32),
                                     _dptr(count, torch.int32), _stream(stream))


def pf_track_frame(vol, depth, intr, params: pf_track_params, init_pose, stream=None):
    """Returns (status, pose 4x4, stats dict)."""
    import torch
    out = (C.c_double * 16)()
    stats = pf_track_stats()
    st = load().pf_track_frame(vol, _dptr(depth, torch.float32), C.byref(intrinsics(intr)), C.byref(params),
                               _pose16(init_pose), out, C.byref(stats), _stream(stream))
    _check(st, "pf_track_frame", ok=(PF_OK, PF_ERR_TRACK_LOST))
    return st, np.array(out[:], dtype=np.float64).reshape(4, 4), stats.to_dict()


def pf_track_frame_async(vol, depth, intr, params: pf_track_params, init_pose_dev, out_pose_dev,
                         stats_dev=None, stream=None) -> int:
    import torch
    return _check(load().pf_track_frame_async(vol, _dptr(depth, torch.float32), C.byref(intrinsics(intr)),
                                              C.byref(params), _dptr(init_pose_dev, torch.float64),
                                              _dptr(out_pose_dev, torch.float64), _dptr(stats_dev),
                                              _stream(stream)), "pf_track_frame_async")


def pf_track_reserve(vol, max_pixels: int, k_max: int) -> int:
    return _check(load().pf_track_reserve(vol, int(max_pixels), int(k_max)), "pf_track_reserve")


def pf_raycast(vol, intr, pose, depth_out, normal_out=None, stream=None) -> int:
    import torch
    return _check(load().pf_raycast(vol, C.byref(intrinsics(intr)), _pose16(pose),
                                    _dptr(depth_out, torch.float32), _dptr(normal_out, torch.float32),
                                    _stream(stream)), "pf_raycast")


def pf_set_fitness_variant(vol, variant: int) -> int:
    return _check(load().pf_set_fitness_variant(vol, int(variant)), "pf_set_fitness_variant")


def pf_volume_info(vol):
    """(storage bytes, cell view) of a volume: -1 no view, 1 full, 2 narrow."""
    b, m = C.c_ulonglong(0), C.c_int(0)
    _check(load().pf_volume_info(vol, C.byref(b), C.byref(m)), "pf_volume_info")
    return int(b.value), int(m.value)


def pf_launch_count() -> int:
    return int(load().pf_launch_count())


def pf_volume_last_error(vol, clear: bool = False) -> int:
    """The last failing status of a call on the volume (PF_OK if none)."""
    return int(load().pf_volume_last_error(vol, 1 if clear else 0))


def pf_alloc_count() -> int:
    """Device allocations the library has made since it was loaded."""
    return int(load().pf_alloc_count())


def pf_gather_probe(buf, n_records: int, mode: int, loads_per_thread: int, out=None, stream=None) -> int:
    """Launch the memory-ceiling probe (mode 0: L2 -> SM stream, 1: scattered
    32-byte records) over `buf` (n_records x 8 float32, on the device);
    returns the thread count (out None: only that, nothing launched)."""
    import torch
    n = C.c_longlong(0)
    _check(load().pf_gather_probe(_dptr(buf, torch.float32), int(n_records), int(mode), int(loads_per_thread),
                                  _dptr(out, torch.float32), C.byref(n), _stream(stream)), "pf_gather_probe")
    return int(n.value)


def pf_set_kernel_timing(enable: bool) -> int:
    return load().pf_set_kernel_timing(1 if enable else 0)


def pf_kernel_timing(kernel_class: str):
    """(total ms, launches) for the class since the last query."""
    ms = C.c_double()
    n = C.c_longlong()
    _check(load().pf_kernel_timing(kernel_class.encode(), C.byref(ms), C.byref(n)), "pf_kernel_timing")
    return ms.value, n.value


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

def track_params(templates_dev, n_iters=20, k_sched=(1024, 3072, 10240), decim_sched=(8, 16, 32),
                 init_rot_deg=10.0, init_trans_cm=10.0, beta=0.1, update_mode=0, compose_mode=0,
                 min_valid_frac=0.0) -> pf_track_params:
    """Search parameters; defaults are the paper's (Sec. III-B, IV-A)."""
    import torch
    if not (templates_dev.is_cuda and templates_dev.dtype == torch.float32 and templates_dev.dim() == 2
            and templates_dev.shape[1] == 6 and templates_dev.is_contiguous()):
        raise ValueError("templates must be a contiguous CUDA float32 tensor of shape (k_max, 6)")
    p = pf_track_params()
    p.n_iters = n_iters
    p.k_sched = (C.c_int * 3)(*k_sched)
    p.decim_sched = (C.c_int * 3)(*decim_sched)
    p.init_rot_deg = init_rot_deg
    p.init_trans_cm = init_trans_cm
    p.beta = beta
    p.templates_dev = templates_dev.data_ptr()
    p.k_max = templates_dev.shape[0]
    p.update_mode = update_mode
    p.compose_mode = compose_mode
    p.min_valid_frac = min_valid_frac
    p._templates_ref = templates_dev  # keep the tensor alive with the struct
    return p


class Volume:
    """A TSDF volume on the current CUDA device (owns pf_volume)."""

    def __init__(self, nx, ny, nz, voxel_size, trunc, origin=(0.0, 0.0, 0.0), max_weight=255, cell_view=0,
                 stream=None, tsdf_dtype=PF_F32, weight_u8=0, search_dtype=PF_F32):
        self.desc = pf_volume_desc(nx, ny, nz, voxel_size, trunc, (C.c_float * 3)(*origin), tsdf_dtype, weight_u8,
                                   max_weight, cell_view, search_dtype)
        self.n_nodes = nx * ny * nz
        self.handle = pf_create_volume(self.desc, stream)

    @classmethod
    def from_grid(cls, grid, max_weight=255, cell_view=0, tsdf_dtype=PF_F32, weight_u8=0, search_dtype=PF_F32):
        return cls(grid.nx, grid.ny, grid.nz, grid.voxel_size, grid.trunc, grid.origin, max_weight, cell_view,
                   tsdf_dtype=tsdf_dtype, weight_u8=weight_u8, search_dtype=search_dtype)

    def close(self):
        if getattr(self, "handle", None):
            pf_destroy_volume(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        pf_reset_volume(self.handle, stream)

    def upload(self, tsdf, weight):
        pf_volume_upload(self.handle, tsdf, weight)

    def download(self):
        return pf_volume_download(self.handle, self.n_nodes)

    def integrate(self, depth, intr, pose, stream=None):
        pf_integrate(self.handle, depth, intr, pose, stream)

    def integrate_async(self, depth, intr, pose_dev, stream=None):
        pf_integrate_async(self.handle, depth, intr, pose_dev, stream)

    def track_frame_async(self, depth, intr, params, init_pose_dev, out_pose_dev, stats_dev=None, stream=None):
        pf_track_frame_async(self.handle, depth, intr, params, init_pose_dev, out_pose_dev, stats_dev, stream)

    def reserve(self, max_pixels, k_max):
        pf_track_reserve(self.handle, max_pixels, k_max)

    def set_fitness_variant(self, variant: int):
        pf_set_fitness_variant(self.handle, variant)

    def info(self) -> dict:
        b, m = pf_volume_info(self.handle)
        return {"storage_bytes": b, "cell_view": m}

    def align_loss(self, points, poses, counts=None, xi=None, dloss=None, grad_xi=False, grad_tsdf=False,
                   stream=None):
        """points: (F, N, 4) float32 CUDA; poses: (F, 4, 4) float64 CUDA ->
        (loss (F,) float64, count (F,) int32, dL/dxi (F, 6) or None,
        dL/dV (n_nodes,) float32 or None)."""
        import torch
        F, N = points.shape[0], points.shape[1]
        dev = points.device
        loss = torch.empty(F, dtype=torch.float64, device=dev)
        cnt = torch.empty(F, dtype=torch.int32, device=dev)
        gx = torch.empty((F, 6), dtype=torch.float64, device=dev) if grad_xi else None
        gv = torch.empty(self.n_nodes, dtype=torch.float32, device=dev) if grad_tsdf else None
        pf_align_loss(self.handle, points, counts, N, F, poses, xi, dloss, loss, cnt, gx, gv, stream)
        return loss, cnt, gx, gv

    def polish(self, points, pose, steps=10, n_dev=None, stream=None):
        """Gauss-Newton polish of pose (16 float64 CUDA, in place) over
        points (N, 4) -> (trace (steps+1,) float64, accepted (1,) int32)."""
        import torch
        trace = torch.empty(steps + 1, dtype=torch.float64, device=pose.device)
        acc = torch.empty(1, dtype=torch.int32, device=pose.device)
        pf_polish(self.handle, points, n_dev, points.shape[0], pose, steps, trace, acc, stream)
        return trace, acc

    def fitness(self, points, poses, stream=None):
        """points: (N, 4) float32 CUDA; poses: (K, 12) float32 CUDA -> (E, C) CUDA tensors."""
        import torch
        k = poses.shape[0]
        E = torch.empty(k, dtype=torch.float32, device=poses.device)
        Cn = torch.empty(k, dtype=torch.int32, device=poses.device)
        pf_fitness(self.handle, points, points.shape[0], poses, k, E, Cn, stream)
        return E, Cn

    def track_frame(self, depth, intr, params, init_pose, stream=None):
        return pf_track_frame(self.handle, depth, intr, params, init_pose, stream)

    def raycast(self, intr, pose, normals=True, stream=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        d = torch.empty((intr.height, intr.width), dtype=torch.float32, device=dev)
        n = torch.empty((intr.height, intr.width, 3), dtype=torch.float32, device=dev) if normals else None
        pf_raycast(self.handle, intr, pose, d, n, stream)
        return d, n


def backproject(depth, intr, stream=None):
    """(points (H*W, 4) CUDA float32, n) -- n valid points at the front."""
    import torch
    pts = torch.empty((intr.width * intr.height, 4), dtype=torch.float32, device=depth.device)
    n = torch.zeros(1, dtype=torch.int32, device=depth.device)
    pf_backproject(depth, intr, pts, n, stream)
    return pts, n


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

def _align_function():
    import torch

    class AlignLoss(torch.autograd.Function):
        """L_f = sum of squared TSDF residuals of frame f at pose
        Exp(omega_f) (R_f x + t_f) + v_f; differentiable in xi = (omega, v)
        and, through `tsdf_sink`, in the volume's stored node values (the
        sink's values are not read; its gradient receives dL/dV)."""

        @staticmethod
        def forward(ctx, xi, tsdf_sink, vol, points, poses, counts):
            loss, cnt, _, _ = vol.align_loss(points, poses, counts=counts, xi=xi.detach().contiguous())
            ctx.vol, ctx.points, ctx.poses, ctx.counts = vol, points, poses, counts
            ctx.save_for_backward(xi)
            ctx.want_v = tsdf_sink is not None and tsdf_sink.requires_grad
            return loss

        @staticmethod
        def backward(ctx, dloss):
            (xi,) = ctx.saved_tensors
            _, _, gx, gv = ctx.vol.align_loss(ctx.points, ctx.poses, counts=ctx.counts,
                                              xi=xi.detach().contiguous(),
                                              dloss=dloss.detach().to(torch.float64).contiguous(),
                                              grad_xi=ctx.needs_input_grad[0], grad_tsdf=ctx.want_v)
            return gx, gv, None, None, None, None

    return AlignLoss


def align_loss(vol, points, poses, xi, counts=None, tsdf_sink=None):
    """Differentiable alignment loss (see AlignLoss).  points (F, N, 4) f32,
    poses (F, 4, 4) f64, xi (F, 6) f64 (requires_grad for dL/dxi)."""
    return _align_function().apply(xi, tsdf_sink, vol, points, poses, counts)


# ---------------------------------------------------------------------------
# batches of sequences
# ---------------------------------------------------------------------------

class _DevArray:
    """A view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class Batch:
    """Independent sequences stepped together (pf_batch_*).  The depth,
    relative-pose, pose and stats buffers are library-owned device memory,
    exposed as torch tensors that alias it."""

    def __init__(self, volumes, cams, params, use_graph=True):
        import torch
        n = len(volumes)
        self._volumes = list(volumes)   # keep the volumes alive
        self._params = list(params)     # and the templates their params point to
        vols = (C.c_void_p * n)(*[v.handle for v in volumes])
        intrs = (pf_intrinsics * n)(*[intrinsics(c) for c in cams])
        prms = (pf_track_params * n)(*params)
        out = C.c_void_p()
        _check(load().pf_batch_create(n, vols, intrs, prms, int(bool(use_graph)), C.byref(out)), "pf_batch_create")
        self.handle = out
        self.n = n
        self.depth, self.rel, self.pose, self.stats = [], [], [], []
        sz = C.sizeof(pf_track_stats)
        for i, intr in enumerate(cams):
            d, r, p, st = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
            _check(load().pf_batch_buffers(out, i, C.byref(d), C.byref(r), C.byref(p), C.byref(st)),
                   "pf_batch_buffers")
            self.depth.append(torch.as_tensor(_DevArray(d.value, (intr.height, intr.width), "<f4"), device="cuda"))
            self.rel.append(torch.as_tensor(_DevArray(r.value, (4, 4), "<f8"), device="cuda"))
            self.pose.append(torch.as_tensor(_DevArray(p.value, (4, 4), "<f8"), device="cuda"))
            self.stats.append(torch.as_tensor(_DevArray(st.value, (sz,), "|u1"), device="cuda"))

    def fuse(self, stream=None):
        _check(load().pf_batch_fuse(self.handle, _stream(stream)), "pf_batch_fuse")

    def step(self, stream=None):
        _check(load().pf_batch_step(self.handle, _stream(stream)), "pf_batch_step")

    def autotune(self, stream=None) -> int:
        c = C.c_int()
        _check(load().pf_batch_autotune(self.handle, _stream(stream), C.byref(c)), "pf_batch_autotune")
        return c.value

    def set_points_per_block(self, p: int):
        _check(load().pf_batch_set_points_per_block(self.handle, int(p)), "pf_batch_set_points_per_block")

    def set_mapping_threshold(self, voxels: float):
        _check(load().pf_batch_set_mapping_threshold(self.handle, float(voxels)), "pf_batch_set_mapping_threshold")

    def tuning(self) -> dict:
        """{"points_per_block": ..., "mapping_threshold": ... (0 = each volume's default)}."""
        p, t = C.c_int(), C.c_float()
        _check(load().pf_batch_tuning(self.handle, C.byref(p), C.byref(t)), "pf_batch_tuning")
        return {"points_per_block": p.value, "mapping_threshold": t.value}

    def stats_dict(self, i: int) -> dict:
        return pf_track_stats.from_buffer_copy(self.stats[i].cpu().numpy().tobytes()).to_dict()

    def close(self):
        if getattr(self, "handle", None):
            load().pf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
