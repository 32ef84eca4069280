"""The C-ABI library loads, exports every declared symbol, and rejects bad
arguments on the host before touching the GPU (no compute calls here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_24236_gb300 import build
    build.build()
    import paper_2509_24236_gb300 as pf
    return pf.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "profusion.h")).read()
    return sorted(set(re.findall(r"PF_API\s+[^;(]*?\b(pf_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pf_create_volume", "pf_integrate", "pf_fitness", "pf_track_frame", "pf_raycast",
                     "pf_destroy_volume", "pf_track_frame_async", "pf_volume_download", "pf_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2509_24236_gb300 import LIB_PATH, EXPORTS
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(pf_\w+)", out))
    for name in declared_symbols():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(EXPORTS) == set(declared_symbols())
    # nothing beyond the declared C ABI leaks out of the library
    assert exported == set(declared_symbols())


def test_status_strings(lib):
    import paper_2509_24236_gb300 as pf
    assert pf.status_string(pf.PF_OK) == "ok"
    assert pf.status_string(pf.PF_ERR_TRACK_LOST) == "tracking lost"
    assert pf.status_string(99) == "unknown status"


def test_host_side_validation_without_a_gpu(lib):
    import paper_2509_24236_gb300 as pf
    out = C.c_void_p()
    # no descriptor / no output pointer
    assert lib.pf_create_volume(None, None, C.byref(out)) == pf.PF_ERR_INVALID_ARG
    good = pf.pf_volume_desc(8, 8, 8, 0.1, 0.3, (C.c_float * 3)(0, 0, 0), pf.PF_F32, 0, 255)
    assert lib.pf_create_volume(C.byref(good), None, None) == pf.PF_ERR_INVALID_ARG
    bad = [
        pf.pf_volume_desc(1, 8, 8, 0.1, 0.3, (C.c_float * 3)(0, 0, 0), pf.PF_F32, 0, 255),
        pf.pf_volume_desc(8, 8, 8, 0.0, 0.3, (C.c_float * 3)(0, 0, 0), pf.PF_F32, 0, 255),
        pf.pf_volume_desc(8, 8, 8, 0.1, -1.0, (C.c_float * 3)(0, 0, 0), pf.PF_F32, 0, 255),
        pf.pf_volume_desc(8, 8, 8, 0.1, 0.3, (C.c_float * 3)(0, float("nan"), 0), pf.PF_F32, 0, 255),
        pf.pf_volume_desc(8, 8, 8, 0.1, 0.3, (C.c_float * 3)(0, 0, 0), pf.PF_F32, 0, 0),
        pf.pf_volume_desc(4096, 4096, 4096, 0.1, 0.3, (C.c_float * 3)(0, 0, 0), pf.PF_F32, 0, 255),
        # cell view modes are -1, 0, 1, 2
        pf.pf_volume_desc(8, 8, 8, 0.1, 0.3, (C.c_float * 3)(0, 0, 0), pf.PF_F32, 0, 255, 3),
        pf.pf_volume_desc(8, 8, 8, 0.1, 0.3, (C.c_float * 3)(0, 0, 0), pf.PF_F16, 0, 255, -2),
    ]
    for d in bad:
        assert lib.pf_create_volume(C.byref(d), None, C.byref(out)) == pf.PF_ERR_INVALID_ARG
    # storage types: f32, f16, bf16 and scaled e4m3 tsdf and uint8 weights
    # exist, other codes do not; a uint8 weight cannot count past 255
    bad_type = pf.pf_volume_desc(8, 8, 8, 0.1, 0.3, (C.c_float * 3)(0, 0, 0), 7, 0, 255)
    assert lib.pf_create_volume(C.byref(bad_type), None, C.byref(out)) == pf.PF_ERR_UNSUPPORTED
    for dt, u8, mw in ((pf.PF_F16, 1, 256), (pf.PF_BF16, 2, 255), (pf.PF_F32, -1, 10)):
        d = pf.pf_volume_desc(8, 8, 8, 0.1, 0.3, (C.c_float * 3)(0, 0, 0), dt, u8, mw)
        assert lib.pf_create_volume(C.byref(d), None, C.byref(out)) == pf.PF_ERR_INVALID_ARG
    # a search view narrower than the storage: float grids only, with a cell
    # view, of a known type
    for dt, view, search, want in ((pf.PF_F16, 0, pf.PF_BF16, pf.PF_ERR_UNSUPPORTED),
                                   (pf.PF_BF16, 1, pf.PF_FP8E4M3, pf.PF_ERR_UNSUPPORTED),
                                   (pf.PF_F32, 0, 9, pf.PF_ERR_UNSUPPORTED),
                                   (pf.PF_F32, -1, pf.PF_F16, pf.PF_ERR_INVALID_ARG)):
        d = pf.pf_volume_desc(8, 8, 8, 0.1, 0.3, (C.c_float * 3)(0, 0, 0), dt, 0, 255, view, search)
        assert lib.pf_create_volume(C.byref(d), None, C.byref(out)) == want, (dt, view, search)
    # NULL volume / pointers
    intr = pf.pf_intrinsics(4, 3, 2.0, 2.0, 1.5, 1.0, 0.1, 8.0)
    pose = (C.c_double * 16)(*[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1])
    assert lib.pf_integrate(None, C.c_void_p(1), C.byref(intr), pose, None) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_fitness(None, None, 0, None, 1, None, None, None) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_raycast(None, C.byref(intr), pose, None, None, None) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_track_frame(None, None, C.byref(intr), None, pose, pose, None, None) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_align_loss(None, None, None, 0, 1, None, None, None, None, None, None, None,
                             None) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_polish(None, None, None, 0, None, 10, None, None, None) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_volume_info(None, None, None) == pf.PF_ERR_INVALID_ARG
    bout = C.c_void_p()
    assert lib.pf_batch_create(0, None, None, None, 1, C.byref(bout)) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_batch_create(1, (C.c_void_p * 1)(None), C.byref(intr), None, 1,
                               C.byref(bout)) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_batch_step(None, None) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_batch_buffers(None, 0, None, None, None, None) == pf.PF_ERR_INVALID_ARG
    bad_intr = pf.pf_intrinsics(0, 3, 2.0, 2.0, 1.5, 1.0, 0.1, 8.0)
    assert lib.pf_backproject(C.c_void_p(1), C.byref(bad_intr), C.c_void_p(1), 100, C.c_void_p(1),
                              None) == pf.PF_ERR_INVALID_ARG
    neg_depth = pf.pf_intrinsics(4, 3, 2.0, 2.0, 1.5, 1.0, -0.1, 8.0)
    assert lib.pf_backproject(C.c_void_p(1), C.byref(neg_depth), C.c_void_p(1), 100, C.c_void_p(1),
                              None) == pf.PF_ERR_INVALID_ARG
    # capacity below width * height
    assert lib.pf_backproject(C.c_void_p(1), C.byref(intr), C.c_void_p(1), 11, C.c_void_p(1),
                              None) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_set_kernel_timing(0) == pf.PF_OK
    ms, n = C.c_double(), C.c_longlong()
    assert lib.pf_kernel_timing(b"nope", C.byref(ms), C.byref(n)) == pf.PF_ERR_INVALID_ARG
    assert lib.pf_kernel_timing(b"fitness", C.byref(ms), C.byref(n)) == pf.PF_OK and n.value == 0
    assert lib.pf_launch_count() == 0


def test_binding_refuses_to_run_without_the_library(tmp_path):
    import paper_2509_24236_gb300 as pf
    with pytest.raises(ImportError):
        pf._lib_backup = pf._lib
        pf._lib = None
        try:
            pf.load(str(tmp_path / "missing.so"))
        finally:
            pf._lib = pf._lib_backup


def test_instrumentation_validation_without_a_gpu(lib):
    import paper_2509_24236_gb300 as pf
    assert lib.pf_volume_last_error(None, 0) == pf.PF_ERR_INVALID_ARG
    n = C.c_longlong(0)
    buf = C.c_void_p(1 << 20)   # never dereferenced: every case below fails host-side checks first
    assert lib.pf_gather_probe(buf, 64, 0, 1, None, None, None) == pf.PF_ERR_INVALID_ARG      # no output count
    assert lib.pf_gather_probe(buf, 64, 2, 1, None, C.byref(n), None) == pf.PF_ERR_INVALID_ARG  # mode
    assert lib.pf_gather_probe(buf, 48, 0, 1, None, C.byref(n), None) == pf.PF_ERR_INVALID_ARG  # not a multiple of 32
    assert lib.pf_gather_probe(buf, 64, 0, 0, None, C.byref(n), None) == pf.PF_ERR_INVALID_ARG  # no loads
    assert lib.pf_gather_probe(C.c_void_p((1 << 20) + 16), 64, 0, 1, None, C.byref(n), None) == \
        pf.PF_ERR_INVALID_ARG                                                                   # misaligned
    assert isinstance(lib.pf_alloc_count(), int)
