"""Boundary behaviour that needs a device: the per-volume record of the last
failing status (kept by every call that takes a volume)."""
import ctypes as C

import pytest

import synth

from gpu_helpers import load_pf, torch_cuda

pytestmark = pytest.mark.gpu


def test_volume_keeps_its_last_failing_status():
    torch = torch_cuda()
    pf = load_pf()
    lib = pf.load()
    vol = pf.Volume.from_grid(synth.ROOM64_GRID)
    assert pf.pf_volume_last_error(vol.handle) == pf.PF_OK
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(64, dtype=torch.int32, device="cuda")
    # k = 0 poses: rejected on the host, nothing enqueued
    st = lib.pf_fitness(vol.handle, C.c_void_p(buf.data_ptr()), 4, C.c_void_p(buf.data_ptr()), 0,
                        C.c_void_p(buf.data_ptr()), C.c_void_p(cnt.data_ptr()), None)
    assert st == pf.PF_ERR_INVALID_ARG
    # a later successful call leaves the record alone
    E, Cn = vol.fitness(buf.view(16, 4), buf[:12].view(1, 12).contiguous())
    torch.cuda.synchronize()
    assert pf.pf_volume_last_error(vol.handle) == pf.PF_ERR_INVALID_ARG
    assert pf.pf_volume_last_error(vol.handle, clear=True) == pf.PF_ERR_INVALID_ARG
    assert pf.pf_volume_last_error(vol.handle) == pf.PF_OK
    # a bad variant is kept too
    assert lib.pf_set_fitness_variant(vol.handle, 99) == pf.PF_ERR_INVALID_ARG
    assert pf.pf_volume_last_error(vol.handle) == pf.PF_ERR_INVALID_ARG
    vol.close()
