"""GPU tests of the warp-blocked passes of a call run in one persistent launch (kernel 4).

Each warp takes (pass, tile) tasks in order and starts one once the tiles around it have finished
the pass before, so passes overlap.  The arithmetic of every tile is that of the launch-per-pass
path (kernel 2), and the energy partials are summed in the same order, so at the same rows per
tile the states and the energies must agree with kernel 2 bit for bit: with and without the
energy, for odd and even pass counts and with leftover steps, on grids from a few tiles to more
tiles than one wave.  With its own rows rule (rows = 0) the tiles differ from kernel 2's, so each
thread's FP32 energy sum covers other nodes and the energies agree to FP32 rounding; the states
still agree bit for bit.  It is also the automatic choice, and must equal the one-step pass.
"""
import numpy as np
import pytest
import torch

from paper_2005_11931_gb300 import inputs, tsu

pytestmark = pytest.mark.gpu

DEPTH = {"background": 1.0, "eps": 0.03, "sings": [(0, 1, 1.0, 0.5, 0.5), (2, 1, 0.01, 0.5, 0.5)]}


def run(nx, ny, steps, kernel, energy, rows=0, seed=3):
    sim = tsu.Simulation.create(nx, DEPTH, dtype="f32", form=tsu.TSU_FORM_INCREMENT, ny=ny)
    rng = np.random.default_rng(seed)
    u0n = inputs.gaussian_hump(nx, ny, sim.g.ld, 0.35, 0.45, 0.07)
    u0n[1:-1, 1:nx - 1] += 0.05 * rng.standard_normal((ny - 2, nx - 2))
    u0 = torch.from_numpy(u0n).float().cuda()
    u1 = torch.zeros_like(u0)
    u1[1:-1, 1:nx - 1] = torch.from_numpy(0.3 * rng.standard_normal((ny - 2, nx - 2))).float()
    sim.init(u0, u1)
    e = torch.zeros(steps, dtype=torch.float64, device="cuda") if energy else None
    sim.step(steps, energy=e, kernel=kernel, rows=rows)
    tsu.tsu_sync_status(sim.ws, sim.ws.numel())
    return sim.u.clone(), sim.v.clone(), (e.clone() if energy else None), sim.state.step


@pytest.mark.parametrize("nx,ny,steps,rows", [
    (257, 257, 40, 16),      # 3 strips x 16 chunks, 10 passes
    (1000, 700, 45, 0),      # ragged, 11 passes and one leftover step
    (130, 2000, 23, 32),     # 2 strips (no inner strip), odd pass count, 3 leftover steps
    (2048, 2048, 400, 0),    # one wave of tiles, 100 passes (more than the energy slots)
    (4096, 1024, 64, 16),    # more tiles than one wave holds warps
])
@pytest.mark.parametrize("energy", [True, False])
def test_persistent_passes_equal_one_launch_per_pass(nx, ny, steps, rows, energy):
    ua, va, ea, sa = run(nx, ny, steps, 4, energy, rows)
    ub, vb, eb, sb = run(nx, ny, steps, 2, energy, rows)
    assert sa == sb
    assert torch.equal(ua, ub) and torch.equal(va, vb)
    if energy:
        if rows:
            assert torch.equal(ea, eb)
        else:
            # each thread's compensated FP32 sum covers other nodes: equal to FP32 rounding
            assert torch.allclose(ea, eb, rtol=1e-6, atol=0.0)
        assert torch.isfinite(ea).all() and (ea > 0).all()


@pytest.mark.parametrize("nx,ny,steps", [(301, 257, 201), (2048, 2048, 61)])
def test_automatic_choice_equals_one_step_passes(nx, ny, steps):
    ua, va, ea, _ = run(nx, ny, steps, 0, True)
    ub, vb, eb, _ = run(nx, ny, steps, 1, True)
    assert torch.equal(ua, ub) and torch.equal(va, vb)
    assert torch.allclose(ea, eb, rtol=1e-6, atol=0.0)  # the one-step pass sums its energy terms otherwise


def test_persistent_pass_refuses_what_it_cannot_do():
    g = tsu.grid(200)
    sim = tsu.Simulation.create(200, DEPTH, dtype="f32", form=tsu.TSU_FORM_STANDARD)
    sim.init(torch.zeros((g.ny, g.ld), dtype=torch.float32, device="cuda"))
    with pytest.raises(tsu.TsuError) as ex:
        sim.step(8, kernel=4)
    assert ex.value.code == tsu.TSU_EINVAL


@pytest.mark.parametrize("energy", [True, False])
def test_persistent_pass_bounded_wait_reports_timeout_and_context_survives(energy):
    """Failure detection without a fault: the test hook keeps tile 0 from ever reporting a pass
    done, so the tasks around it wait until their bounded wait (20 ms) expires.  The status word
    then says TSU_ETIMEOUT, every warp leaves, and the next call on the same context works and
    equals the launch-per-pass path."""
    n, steps = 600, 40
    sim = tsu.Simulation.create(n, DEPTH, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
    u0 = torch.from_numpy(inputs.gaussian_hump(n, n, sim.g.ld, 0.3, 0.5, 0.05)).float().cuda()
    sim.init(u0)
    e = torch.zeros(steps, dtype=torch.float64, device="cuda") if energy else None
    sim.step(steps, energy=e, kernel=4, rows=16, debug=2)
    with pytest.raises(tsu.TsuError) as ei:
        tsu.tsu_sync_status(sim.ws, sim.ws.numel())
    assert ei.value.code == tsu.TSU_ETIMEOUT
    # the status was cleared and the context is usable
    ua, va, _, _ = run(n, n, steps, 4, energy, 16)
    ub, vb, _, _ = run(n, n, steps, 2, energy, 16)
    assert torch.equal(ua, ub) and torch.equal(va, vb)
