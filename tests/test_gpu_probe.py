"""pf_gather_probe, the memory-ceiling probe behind the fitness kernel's
roofline: it must read exactly the records its documented position sequence
names (so that bytes / time is a rate of real loads), checked by recomputing
every thread's sum on the host."""
import numpy as np
import pytest

from gpu_helpers import load_pf, torch_cuda

pytestmark = pytest.mark.gpu


def _mix(x):
    x = x.astype(np.uint64)
    m = np.uint64(0xFFFFFFFF)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x85EBCA6B)) & m
    x ^= x >> np.uint64(13)
    x = (x * np.uint64(0xC2B2AE35)) & m
    x ^= x >> np.uint64(16)
    return x


def _expected(vals, n_rec, mode, loads, threads):
    tid = np.arange(threads, dtype=np.uint64)
    h = _mix(tid >> np.uint64(5) if mode == 0 else tid)
    lane = tid & np.uint64(31)
    acc = np.zeros(threads, dtype=np.float64)
    rec_sum = vals.reshape(n_rec, 8).sum(axis=1)  # small integers: every float sum is exact
    for _ in range(loads):
        h = (h * np.uint64(1664525) + np.uint64(1013904223)) & np.uint64(0xFFFFFFFF)
        if mode == 0:
            rec = ((h * np.uint64(n_rec // 32)) >> np.uint64(32)) * np.uint64(32) + lane
        else:
            rec = (h * np.uint64(n_rec)) >> np.uint64(32)
        acc += rec_sum[rec.astype(np.int64)]
    return acc


@pytest.mark.parametrize("mode", [0, 1])
def test_probe_reads_the_documented_records(mode):
    torch = torch_cuda()
    pf = load_pf()
    n_rec, loads = 4096, 5
    rng = np.random.default_rng(3 + mode)
    vals = rng.integers(0, 16, size=n_rec * 8).astype(np.float32)
    buf = torch.from_numpy(vals).cuda()
    threads = pf.pf_gather_probe(buf, n_rec, mode, loads)
    out = torch.full((threads,), -1.0, device="cuda")
    assert pf.pf_gather_probe(buf, n_rec, mode, loads, out) == threads
    got = out.cpu().numpy().astype(np.float64)
    assert np.array_equal(got, _expected(vals, n_rec, mode, loads, threads))


def test_probe_rejects_bad_sizes():
    torch = torch_cuda()
    pf = load_pf()
    buf = torch.zeros(8 * 64, device="cuda")
    out = torch.zeros(1 << 20, device="cuda")
    for n_rec, mode, loads in ((33, 0, 1), (16, 1, 1), (64, 2, 1), (64, 0, 0)):
        with pytest.raises(pf.ProfusionError):
            pf.pf_gather_probe(buf, n_rec, mode, loads, out)
