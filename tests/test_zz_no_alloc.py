"""The allocation-free field sum (wfa_sum_f32_noalloc), for callers that cannot
allocate device memory: through the C ABI it must agree with the total-heat
reduction of a grid holding the same field (which sums with scratch the grid
allocated), on two calls in a row.

The tests here depend on no other test and pass alone in a fresh process as
well as after the rest of the suite. The file name only makes pytest collect
it last, so that a run stopping at the first failure (-x) has run every other
test before it reaches this one."""
import ctypes

import numpy as np
import pytest

import paper_2209_13768_gb300 as wfa

pytestmark = pytest.mark.gpu


def _field(seed, shape):
    nx, ny, nz = shape
    return np.random.default_rng(seed).uniform(-1, 2, (nz, ny, nx)).astype(np.float32)


def test_sum_noalloc_matches_total_heat_twice():
    torch = pytest.importorskip("torch")
    shape = (97, 61, 45)
    h = (0.5, 1.25, 2.0)
    vol = h[0] * h[1] * h[2]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (1, 2):   # two calls in a row, different fields
        T = _field(seed, shape)
        with wfa.Grid(shape, h=h) as g:
            g.set_field(T)
            ref = g.total_heat()
        x = torch.from_numpy(T.ravel()).cuda()
        torch.cuda.synchronize()
        wfa.sum_f32_noalloc(x.data_ptr(), x.numel(), vol, out.data_ptr())
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (seed, got, ref)
        assert abs(got - float(T.astype(np.float64).sum()) * vol) <= 1e-12 * abs(ref)


def test_sum_noalloc_rejects_sizes_beyond_its_scratch():
    L = wfa.lib()
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    assert L.wfa_sum_f32_noalloc(dummy, (1 << 27) + 1, 1.0, dummy, None) == -1
    assert "maximum" in wfa.last_error()
