"""The forward kernels' exact warp sum on the device (pq_fixsum_device)
against its host twin (pq_fixsum_host), whose arithmetic the CPU tests pin
against exact rationals: the same bits on every lane, for random, cancelling,
spread and tiny inputs and partial warps; a non-finite lane value gives a
non-finite sum."""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2403_04006_gb300 import pq  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pq.load_library()
    return torch.device("cuda:0")


def host_sum(hi, lo):
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    out = np.zeros(2)
    rc = pq.load_library().pq_fixsum_host(hi.ctypes.data_as(ctypes.c_void_p),
                                          lo.ctypes.data_as(ctypes.c_void_p), len(hi),
                                          out.ctypes.data_as(ctypes.c_void_p))
    assert rc == 0
    return out


def device_sum(hi, lo, dev):
    h = torch.tensor(np.asarray(hi, dtype=np.float64), device=dev)
    lw = torch.tensor(np.asarray(lo, dtype=np.float64), device=dev)
    out = torch.full((64,), float("nan"), dtype=torch.float64, device=dev)
    rc = pq.load_library().pq_fixsum_device(h.data_ptr() if h.numel() else None,
                                            lw.data_ptr() if lw.numel() else None, len(hi),
                                            out.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    return out.cpu().numpy().reshape(32, 2)


def cases():
    rng = np.random.default_rng(1234)
    out = []
    for n in (32, 31, 17, 1, 0):
        hi = rng.standard_normal(n) * 2.0 ** rng.integers(-30, 30, n)
        lo = hi * 2.0 ** -53 * rng.uniform(-1, 1, n)
        out.append((f"random{n}", hi, lo))
    hi = rng.standard_normal(32)
    hi[16:] = -hi[:16] * (1 + 2.0 ** -45)
    out.append(("cancel", hi, hi * 2.0 ** -60))
    hi = rng.standard_normal(32) * 2.0 ** rng.integers(-120, 0, 32)
    out.append(("spread", hi, np.zeros(32)))
    hi = rng.standard_normal(32) * 1e-300
    out.append(("tiny", hi, hi * 2.0 ** -53))
    hi = rng.standard_normal(32) * 1e300
    out.append(("huge", hi, np.zeros(32)))
    return out


@pytest.mark.parametrize("name,hi,lo", cases(), ids=[c[0] for c in cases()])
def test_device_sum_matches_the_host_twin_bit_for_bit(dev, name, hi, lo):
    got = device_sum(hi, lo, dev)
    want = host_sum(hi, lo)
    for q in range(32):  # every lane holds the sum
        assert got[q].view(np.int64).tolist() == want.view(np.int64).tolist(), (name, q)


def test_non_finite_lane_gives_a_non_finite_sum(dev):
    hi = np.ones(32)
    hi[7] = math.inf
    got = device_sum(hi, np.zeros(32), dev)
    assert not np.isfinite(got[0, 0])
    hi[7] = math.nan
    got = device_sum(hi, np.zeros(32), dev)
    assert not np.isfinite(got[0, 0])
