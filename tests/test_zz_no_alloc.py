"""tsu_step_n_noalloc: the stepping entry point for callers that cannot allocate device memory.

It must give what tsu_step_n gives with a caller workspace (same one-step pass, same energy), on
two calls in a row (the fixed scratch array is shared between calls and keeps the last call's
contents).  Its refusal of grids the fixed scratch cannot hold is checked without a device
(tests/test_abi.py).  This file is collected last.
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
