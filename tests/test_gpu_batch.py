"""GPU tests of the batched eps-family launch (tsu_batch_run)."""
import numpy as np
import pytest
import torch

from paper_2005_11931_gb300 import inputs, tsu
from tests.gpu_helpers import relerr, run_oracle

pytestmark = pytest.mark.gpu


def family(steps, sizes=(129, 200, 257, 300), count_eps=3):
    return inputs.batched_family(steps=steps, count_eps=count_eps, sizes=sizes)


def make_sims(probs, form):
    sims = []
    for p in probs:
        sim = tsu.Simulation.create(p.n, p.depth, dtype="f32", form=form)
        sim.init(torch.from_numpy(p.initial(sim.g.ld, np.float32)).cuda())
        sims.append(sim)
    return sims


@pytest.mark.parametrize("form", [tsu.TSU_FORM_INCREMENT, tsu.TSU_FORM_STANDARD])
@pytest.mark.parametrize("kernel,K", [(3, 4), (3, 8), (2, 2), (2, 4)])
def test_batched_equals_sequential_bitwise(form, kernel, K):
    probs = family(steps=1 + 5 * K + 3)
    steps = [p.steps - 1 for p in probs]
    seq = make_sims(probs, form)
    for sim, n in zip(seq, steps):
        sim.step(n, kernel=kernel, tdepth=K, rows=64)
    bat = make_sims(probs, form)
    wsb = tsu.tsu_batch_workspace(bat, steps, tdepth=K, rows=64, kernel=kernel)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    tsu.tsu_batch_run(bat, steps, ws, wsb, tdepth=K, rows=64, kernel=kernel)
    tsu.tsu_sync_status(ws, wsb)
    for a, b in zip(seq, bat):
        assert a.state.step == b.state.step
        assert torch.equal(a.u, b.u)
        assert torch.equal(a.bufs[a.state.aux], b.bufs[b.state.aux])


def test_batched_uneven_step_counts():
    probs = family(steps=40)
    rng = np.random.default_rng(3)
    steps = [int(s) for s in rng.integers(0, 60, size=len(probs))]
    seq = make_sims(probs, tsu.TSU_FORM_INCREMENT)
    for sim, n in zip(seq, steps):
        sim.step(n, kernel=2, tdepth=4, rows=64) if n >= 4 else sim.step(n, kernel=1)
    bat = make_sims(probs, tsu.TSU_FORM_INCREMENT)
    wsb = tsu.tsu_batch_workspace(bat, steps, tdepth=4, rows=64)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    tsu.tsu_batch_run(bat, steps, ws, wsb, tdepth=4, rows=64)
    for a, b, n in zip(seq, bat, steps):
        assert b.state.step == 1 + n
        assert torch.equal(a.u, b.u), n


def test_batched_problem_matches_oracle():
    probs = family(steps=1 + 8 * 6 + 2, sizes=(200, 257), count_eps=2)
    steps = [p.steps - 1 for p in probs]
    bat = make_sims(probs, tsu.TSU_FORM_INCREMENT)
    wsb = tsu.tsu_batch_workspace(bat, steps)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    tsu.tsu_batch_run(bat, steps, ws, wsb)
    for p, sim in zip(probs, bat):
        orc = run_oracle(p.n, p.depth, p.initial(), p.steps, energy=False)
        assert relerr(sim.u[:, : p.n].double().cpu().numpy(), orc["u"]) <= 1e-5, p.name


def test_graph_launch_equals_stream_launch():
    """The whole call captured into one CUDA graph (uneven step counts, so blocked rounds of
    shrinking tile prefixes and single leftover steps are all in the graph)."""
    probs = family(steps=40)
    rng = np.random.default_rng(8)
    steps = [int(s) for s in rng.integers(0, 60, size=len(probs))]
    a = make_sims(probs, tsu.TSU_FORM_INCREMENT)
    b = [s.clone() for s in a]
    wsb = tsu.tsu_batch_workspace(a, steps)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    tsu.tsu_batch_run(a, steps, ws, wsb)
    ws2 = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())  # after every allocation and fill above
    with torch.cuda.stream(side):
        tsu.tsu_batch_run(b, steps, ws2, wsb, graph=True, stream=side)
    side.synchronize()
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert (x.state.cur, x.state.aux, x.state.step) == (y.state.cur, y.state.aux, y.state.step)
        assert torch.equal(x.u, y.u)
        assert torch.equal(x.bufs[x.state.aux], y.bufs[y.state.aux])


def test_graph_launch_needs_a_stream():
    probs = family(steps=9)
    sims = make_sims(probs, tsu.TSU_FORM_INCREMENT)
    steps = [8] * len(sims)
    wsb = tsu.tsu_batch_workspace(sims, steps)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    with pytest.raises(tsu.TsuError) as e:
        tsu.tsu_batch_run(sims, steps, ws, wsb, graph=True, stream=0)
    assert e.value.code == tsu.TSU_EINVAL


def test_autotuned_choices_keep_the_results(tmp_path):
    from paper_2005_11931_gb300 import autotune

    cache = autotune.Cache(str(tmp_path / "tune.json"))
    probs = family(steps=50)
    sims = make_sims(probs, tsu.TSU_FORM_INCREMENT)
    ref = [s.clone() for s in sims]
    c = autotune.tune_batch(sims, steps=16, cache=cache)
    assert isinstance(c, autotune.Choice)
    # tuning ran on scratch copies: the states did not move
    for x, y in zip(sims, ref):
        assert x.state.step == y.state.step and torch.equal(x.u, y.u)
    assert autotune.tune_batch(sims, cache=cache) == c  # cached
    steps = [p.steps - 1 for p in probs]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        used = tsu.batch_run(sims, steps, tune=True, cache=cache, stream=side)
    side.synchronize()
    assert used == c.batch_opts(sims)
    for s, n in zip(ref, steps):
        s.step(n, kernel=1)
    torch.cuda.synchronize()
    for x, y in zip(sims, ref):
        assert torch.equal(x.u, y.u)
    # one problem: the tuned stepping choice
    big = tsu.Simulation.create(1025, probs[0].depth, dtype="f32")
    big.init(torch.from_numpy(inputs.gaussian_hump(1025, 1025, big.g.ld, 0.4, 0.5, 0.03, 1.0, np.float32)).cuda())
    other = big.clone()
    cs = autotune.tune_step(big, steps=16, cache=cache)
    big.step(37, kernel=cs.kernel, tdepth=cs.tdepth, rows=cs.rows)
    other.step(37, kernel=1)
    torch.cuda.synchronize()
    assert torch.equal(big.u, other.u)


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("scaled", [False, True])
def test_batch_packing_keeps_the_results(order, scaled):
    """Every tile-table order, with uniform or size-scaled rows per chunk (uneven step counts, so
    that the launches cover shrinking prefixes of the table): the same bits as each problem run
    on its own, one step per pass."""
    probs = family(steps=60, sizes=(129, 200, 257, 300, 521))
    rng = np.random.default_rng(5)
    steps = [int(s) for s in rng.integers(8, 60, size=len(probs))]
    bat = make_sims(probs, tsu.TSU_FORM_INCREMENT)
    rpp = [max(16, (7 * s.g.ny) // 40) for s in bat] if scaled else None
    used = tsu.batch_run(bat, steps, rows=48, order=order, rows_per_problem=rpp)
    assert used["order"] == order
    seq = make_sims(probs, tsu.TSU_FORM_INCREMENT)
    for sim, n in zip(seq, steps):
        sim.step(n, kernel=1)
    torch.cuda.synchronize()
    for a, b, n in zip(seq, bat, steps):
        assert b.state.step == 1 + n
        assert torch.equal(a.u, b.u), n
        assert torch.equal(a.v, b.v), n
