"""Autotuner for the blocked passes: picks, by timing on the caller's own problems, the pass
(warp-blocked, launched per pass or all passes in one persistent launch, or CTA-blocked), its
temporal depth (steps per HBM pass), the rows per tile and, for
the batched family, how the tiles are packed (tile-table order, rows scaled with each problem's
size) and whether to launch through one CUDA graph.  Results are cached per problem
signature (grid shapes, form, GPU name) in a JSON file.

The timed runs advance scratch copies of the simulations (``Simulation.clone``), never the
caller's states, so tuning changes no result; the choice cannot change one either, because every
pass rounds each operation the same way.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import asdict, dataclass

import torch

from . import tsu


@dataclass(frozen=True)
class Choice:
    kernel: int   # 1 one step per pass, 2 warp-blocked, 3 CTA-blocked, 4 warp-blocked in one persistent launch
    tdepth: int   # steps per pass (0: the kernel's default)
    rows: int     # rows per tile (0: the library's rule)
    graph: bool = False
    order: int = 0        # batched tile-table order (tsu_batch_opts.order)
    size_rows: bool = False  # batched: rows per chunk scaled with each problem's size (rows for the largest)

    def rows_per_problem(self, sims):
        """Per-problem rows of a size-scaled packing: ``rows`` for the largest grid, in proportion
        to the row count below it (at least 16), so that every problem's chunks take about as
        long; None for a uniform packing."""
        if not self.size_rows or self.rows == 0:
            return None
        nmax = max(s.g.ny for s in sims)
        return [max(16, int(round(self.rows * s.g.ny / nmax))) for s in sims]

    def batch_opts(self, sims) -> dict:
        """Keyword arguments of tsu.tsu_batch_run for this choice."""
        return dict(tdepth=self.tdepth, rows=self.rows, kernel=self.kernel, graph=self.graph, order=self.order,
                    rows_per_problem=self.rows_per_problem(sims))


def batch_candidates() -> list[Choice]:
    """Configurations tried for a batched family: the pass and its depth, rows per chunk, the
    packing of the tile table (order, size-scaled rows) and the graph launch."""
    out = []
    for rows in (0, 64, 96, 128, 192):
        for graph in (False, True):
            out.append(Choice(2, 4, rows, graph))
    for order in (1, 2):
        for rows in (0, 64, 96):
            out.append(Choice(2, 4, rows, False, order))
    for rows in (64, 96, 128):
        for order in (0, 2):
            out.append(Choice(2, 4, rows, False, order, True))
    out += [Choice(2, 2, 128, False), Choice(3, 8, 128, False), Choice(3, 4, 128, False)]
    return out


def step_candidates() -> list[Choice]:
    """Configurations tried for one problem (FP32, four state buffers, no per-step traces); the
    persistent pass (kernel 4) only runs in the increment form, and is skipped otherwise."""
    out = [Choice(1, 0, 0)]
    for rows in (0, 32, 64, 96, 160):
        out.append(Choice(2, 4, rows))
    for rows in (0, 16, 32, 48, 96):
        out.append(Choice(4, 0, rows))
    out += [Choice(2, 2, 0), Choice(3, 8, 128), Choice(3, 4, 128)]
    return out


def signature(kind: str, sims) -> str:
    shapes = sorted((s.g.nx, s.g.ny, s.g.ld) for s in sims)
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return json.dumps({"kind": kind, "dev": dev, "dtype": sims[0].dtype, "form": sims[0].form, "shapes": shapes})


class Cache:
    """JSON file of signature -> Choice (path: argument, else $TSU_TUNE_CACHE, else
    ~/.cache/tsu/autotune.json)."""

    def __init__(self, path: str | None = None):
        self.path = path or os.environ.get("TSU_TUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "tsu", "autotune.json")
        self.table = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.table = json.load(f)
            except (OSError, ValueError):
                self.table = {}

    def get(self, key: str) -> Choice | None:
        v = self.table.get(key)
        return Choice(**v) if v else None

    def put(self, key: str, choice: Choice) -> None:
        self.table[key] = asdict(choice)
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def wall_timer(fn) -> float:
    """Milliseconds of one call of ``fn`` including all the GPU work it enqueues (the device is
    synchronised before and after; host-side preparation such as descriptor uploads counts)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    return 1e3 * (time.perf_counter() - t0)


def pick(candidates, run, timer=wall_timer, repeats: int = 2) -> tuple[Choice, dict]:
    """The candidate with the least time: each is run once untimed, then ``repeats`` times timed
    (the minimum counts).  Candidates that the library refuses are skipped."""
    times = {}
    for c in candidates:
        try:
            run(c)
        except tsu.TsuError:
            continue
        times[c] = min(timer(lambda: run(c)) for _ in range(repeats))
    if not times:
        raise RuntimeError("no candidate configuration ran")
    best = min(times, key=lambda c: times[c])
    return best, times


def tune_batch(sims, steps: int = 32, cache: Cache | None = None, timer=wall_timer, stream=None) -> Choice:
    """Best configuration of tsu_batch_run for these simulations (FP32, nbuf 4), timing ``steps``
    steps of scratch copies per candidate (the same for every candidate, whatever its depth:
    a multiple of 8 keeps every depth's passes full)."""
    cache = cache if cache is not None else Cache()
    key = signature("batch", sims)
    hit = cache.get(key)
    if hit is not None:
        return hit
    scratch = [s.clone() for s in sims]
    side = stream or torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())  # the clones are made on the current stream
    work = {}  # per candidate: step counts and workspace, made before any timing

    def run(c: Choice):
        o = c.batch_opts(scratch)
        if c not in work:
            nsteps = [steps] * len(scratch)
            wsb = tsu.tsu_batch_workspace(scratch, nsteps, **{key: v for key, v in o.items() if key != "graph"})
            work[c] = (nsteps, torch.zeros(wsb, dtype=torch.uint8, device="cuda"), wsb)
        nsteps, ws, wsb = work[c]
        side.wait_stream(torch.cuda.current_stream())  # the workspace is zeroed on the current stream
        with torch.cuda.stream(side):
            tsu.tsu_batch_run(scratch, nsteps, ws, wsb, stream=side, **o)
        side.synchronize()

    best, _ = pick(batch_candidates(), run, timer)
    cache.put(key, best)
    return best


def tune_step(sim, steps: int = 64, cache: Cache | None = None, timer=wall_timer) -> Choice:
    """Best (kernel, tdepth, rows) of tsu_step_n for this simulation, timing ``steps`` steps of a
    scratch copy with the energy recorded every step."""
    cache = cache if cache is not None else Cache()
    key = signature("step", [sim])
    hit = cache.get(key)
    if hit is not None:
        return hit
    scratch = sim.clone()
    energy = torch.zeros(steps, dtype=torch.float64, device="cuda")

    def run(c: Choice):
        scratch.step(steps, energy=energy, kernel=c.kernel, rows=c.rows, tdepth=c.tdepth)

    best, _ = pick(step_candidates(), run, timer)
    cache.put(key, best)
    return best
