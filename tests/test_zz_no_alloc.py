"""tsu_step_n_noalloc: the stepping entry point for callers that cannot allocate device memory.

It must give what tsu_step_n gives with a caller workspace (same one-step pass, same energy), on
two calls in a row (the fixed scratch array is shared between calls and keeps the last call's
contents), and refuse grids its fixed scratch cannot hold.  This file is collected last.
"""
import numpy as np
import pytest
import torch

from paper_2005_11931_gb300 import inputs, tsu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,form", [("f32", tsu.TSU_FORM_INCREMENT), ("f64", tsu.TSU_FORM_STANDARD)])
def test_noalloc_matches_workspace_entry_point_on_two_calls(dtype, form):
    n = 777
    depth = dict(background=1.0, eps=0.02, mollifier=0, sings=[(0, 1, 1.0, 0.5, 0.5), (2, 1, 0.01, 0.4, 0.6)])
    ref = tsu.Simulation.create(n, depth, dtype=dtype, form=form, nbuf=3)
    na = tsu.Simulation.create(n, depth, dtype=dtype, form=form, nbuf=3)
    u0 = torch.from_numpy(inputs.gaussian_hump(n, n, ref.g.ld, 0.3, 0.45, 0.05)).to(ref.hx.dtype).cuda()
    ref.init(u0)
    na.init(u0)
    e_ref = torch.zeros(90, dtype=torch.float64, device="cuda")
    e_na = torch.full((90,), -1.0, dtype=torch.float64, device="cuda")
    for a, b in ((0, 50), (50, 90)):  # two calls in a row
        # the same pass with the same CTA partition (32 rows per CTA, which the fixed scratch is sized for)
        ref.step(b - a, energy=e_ref[a:b], kernel=1, rows=32)
        tsu.tsu_step_n_noalloc(na.g, na.dtype, na.tau, na.medium, na.state, b - a, energy=e_na[a:b])
        torch.cuda.synchronize()
        assert na.state.step == ref.state.step
        np.testing.assert_allclose(na.u.double().cpu().numpy(), ref.u.double().cpu().numpy(), rtol=0, atol=1e-12)
        np.testing.assert_allclose(na.bufs[na.state.aux].double().cpu().numpy(),
                                   ref.bufs[ref.state.aux].double().cpu().numpy(), rtol=0, atol=1e-12)
        np.testing.assert_allclose(e_na[a:b].cpu().numpy(), e_ref[a:b].cpu().numpy(), rtol=1e-12, atol=0)


def test_noalloc_refuses_grids_beyond_its_fixed_scratch():
    # FP64 on 32800 x 32800 would need ceil(32800/256) * ceil(32798/32) = 129 * 1025 > 65536 partials;
    # the call is refused before any device work, so small dummy buffers suffice
    g = tsu.Grid(32800, 32800, 32800, 1 / 32799, 1 / 32799)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    med = tsu.Medium(buf.data_ptr(), buf.data_ptr(), 1.0, 1.0)
    st = tsu.State()
    for k in range(2):
        st.buf[k] = buf.data_ptr()
    st.buf[1] = buf.data_ptr() + 64
    st.nbuf, st.form, st.cur, st.aux = 2, tsu.TSU_FORM_STANDARD, 1, 0
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_step_n_noalloc(g, "f64", 1e-6, med, st, 1, energy=e)
    assert ei.value.code == tsu.TSU_ENOMEM
    assert "too large" in str(ei.value)
