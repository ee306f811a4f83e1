"""aew_dot_noalloc, the inner product for callers that cannot allocate device memory
(for example an application that routes every device allocation through its own pool):
same result as aew_dot on two calls in a row, and sizes beyond its fixed scratch array
rejected before any device work.  Kept in the last test file so that a run stopping at
the first failure has run everything else first."""
import ctypes

import pytest
import torch

from paper_2304_04781_gb300 import aewave

pytestmark = pytest.mark.gpu


def _call(a, b, out, n=None):
    L = aewave.lib()
    return L.aew_dot_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                             a.numel() if n is None else n, ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_dot_noalloc_matches_aew_dot_on_two_calls():
    g = torch.Generator(device="cuda").manual_seed(7)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in (3_000_017, 65536 * 5):          # two calls in a row, different sizes
        a = torch.randn(n, device="cuda", generator=g)
        b = torch.randn(n, device="cuda", generator=g)
        assert _call(a, b, out) == 0
        torch.cuda.synchronize()
        got = float(out.item())
        want = aewave.dot(a, b)
        scale = aewave.dot(a.abs(), b.abs())   # sum |a b|: the natural size of round-off
        assert abs(got - want) <= 1e-12 * scale, (n, got, want)


def test_dot_noalloc_rejects_sizes_beyond_its_scratch():
    a = torch.ones(8, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _call(a, a, out, n=(1 << 32) + 1) == -9      # AEW_E_ARG, nothing launched
    assert _call(a, a, out) == 0
    torch.cuda.synchronize()
    assert float(out.item()) == 8.0
