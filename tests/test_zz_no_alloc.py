"""The allocation-free weighted sum (vof_volume_sum_noalloc) against the
context's own volume sum (vof_get_stats), through the C-ABI.

Collected last on purpose: it exercises the library's shared scratch array,
so every other test has run before it if it fails under -x. It must pass
both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative, as the FP64 volume checks of the parity tests


@pytest.fixture(scope="module")
def vof():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01524_gb300 import build, vof as V
    build.build()
    return V


def test_noalloc_sum_matches_context_volume_twice(vof):
    import torch
    m = I.hex_mesh(40)
    F0 = I.init_fraction(m, I.sphere((0.35, 0.35, 0.35), 0.15), levels=3)
    ctx = vof.Context(m)
    w = torch.from_numpy(ctx.geometry()["cell_vol"]).cuda()
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    # two calls in a row on different data and sizes: the second must not
    # see anything the first left in the shared scratch
    cases = [(F0, m["n_cell"]), (np.clip(1.7 * F0, 0.0, 1.0)[: 20000], 20000)]
    for F, n in cases:
        ctx_ref = vof.Context(m)
        full = np.zeros(m["n_cell"])
        full[:n] = F[:n]
        ctx_ref.set_fraction(full)
        expected = ctx_ref.stats()["volume"]  # existing entry point
        Fd = torch.from_numpy(np.ascontiguousarray(F[:n])).cuda()
        st = vof.volume_sum_noalloc(w, Fd, out, n=n)
        assert st == vof.VOF_OK, vof.lib().vof_last_error()
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - expected) <= TOL * abs(expected), (got, expected)


def test_noalloc_rejects_sizes_beyond_its_scratch(vof):
    import torch
    w = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = vof.volume_sum_noalloc(w, w, out, n=65536 * 4096 + 1)
    assert st == vof.VOF_EINVAL
    assert b"outside" in vof.lib().vof_last_error()
    assert vof.volume_sum_noalloc(w, w, out, n=-1) == vof.VOF_EINVAL
