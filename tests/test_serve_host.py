"""Host logic of the serving loop (paper_1812_05401_gb300/serve.py) on the CPU.

The loop's device calls are replaced by fakes that record what it asks for:
the binding (solver creation, footprints, grouped steps, the asynchronous
force read) and PyTorch's event and pinned-memory calls. What is checked is
the scheduling itself: rounds of min(remaining, round_steps) steps, FIFO
admission against the memory budget and the slot limit, refusal of requests
that cannot fit or cannot be created, a diverging solve failing alone, every
request answered once with its own force series, and the report's figures.
The GPU tests (test_serve.py) run the same loop on the real library.
"""
import types

import numpy as np
import pytest

from paper_1812_05401_gb300 import inputs as I
from paper_1812_05401_gb300 import serve as S
from paper_1812_05401_gb300 import vplbm as V

BYTES_PER_NODE = 100


class FakeLib:
    """Stands in for the binding: a solver is a record of its step count."""

    VplbmError = V.VplbmError

    def __init__(self, fail_create=(), diverge=()):
        self.fail_create = set(fail_create)
        self.diverge = set(diverge)
        self.solvers = {}
        self.rounds = []        # per grouped step: [(name, steps)]
        self.created = []       # names in creation order
        self.live_bytes = 0
        self.peak_bytes = 0
        self.time = 0.0         # fake clock: 1 ms per grouped step
        lib = self

        class Solver:
            def __init__(s, cfg, bodies, perturbation=None):
                if cfg.w.name in lib.fail_create:
                    raise V.VplbmError(V.VPLBM_ERR_NOMEM, "out of device memory")
                s.w, s.t, s.h = cfg.w, 0, len(lib.solvers) + 1
                lib.solvers[s.h] = s
                lib.created.append(s.w.name)
                lib.live_bytes += lib.vplbm_footprint_bytes(cfg)
                lib.peak_bytes = max(lib.peak_bytes, lib.live_bytes)

            def close(s):
                lib.live_bytes -= s.w.nx * s.w.ny * BYTES_PER_NODE

            def populations(s):
                return np.full((9, s.w.ny, s.w.nx), float(s.t))

            def synchronize(s):
                if s.w.name in lib.diverge:
                    raise V.VplbmError(V.VPLBM_ERR_DIVERGED, "diverged")

        self.Solver = Solver

    def config_from_workload(self, w, ring_len=4096, stream=None, reduce_mass=True, tile_rows=0):
        assert ring_len >= w.steps  # the whole force series fits the ring
        return types.SimpleNamespace(w=w), list(w.bodies)

    def vplbm_footprint_bytes(self, cfg):
        return cfg.w.nx * cfg.w.ny * BYTES_PER_NODE

    def vplbm_group_step(self, handles, steps):
        self.rounds.append([(self.solvers[h].w.name, k) for h, k in zip(handles, steps)])
        for h, k in zip(handles, steps):
            self.solvers[h].t += k
        self.time += 1e-3 * max(steps)

    def vplbm_forces_async(self, h, rec):
        """The records of every step run so far (the ring holds them all)."""
        s = self.solvers[h]
        assert rec.shape == (max(1, s.t), 3)
        rec[:s.t, 0] = np.arange(s.t) + 1000.0 * s.w.seed
        rec[:s.t, 1] = -rec[:s.t, 0]
        rec[:s.t, 2] = 1.0
        return s.t


def fake_torch(gpu_done: bool):
    """Events report the GPU done at once (gpu_done) or only when waited on."""

    class Event:
        def record(self, stream):
            pass

        def query(self):
            return gpu_done

        def synchronize(self):
            pass

    def empty(shape, dtype=None, pin_memory=False):
        a = np.zeros(shape, dtype=np.float64)
        return types.SimpleNamespace(numpy=lambda: a)

    return types.SimpleNamespace(float64=np.float64, empty=empty,
                                 cuda=types.SimpleNamespace(Event=Event))


def workload(name, nx, ny, steps, seed):
    return types.SimpleNamespace(name=name, nx=nx, ny=ny, steps=steps, storage="f32",
                                 collision="mrt", u_ref=0.05, bc="channel", perturbation=0.0,
                                 seed=seed, bodies=[])


def serve(monkeypatch, reqs, budget, gpu_done=True, realtime=False, log=None, fake_clock=False,
          **kw):
    lib = FakeLib(kw.pop("fail_create", ()), kw.pop("diverge", ()))
    monkeypatch.setattr(S, "V", lib)
    if fake_clock:
        kw["clock"] = lambda: lib.time
    srv = S.Server(budget, stream=object(), **kw)
    srv.torch = fake_torch(gpu_done)
    results, rep = srv.run(reqs, realtime=realtime, log=log)
    return lib, srv, {r.name: r for r in results}, rep


def _check_series(r, w):
    assert r.steps == w.steps and len(r.fx) == w.steps
    assert np.array_equal(r.fx, np.arange(w.steps) + 1000.0 * w.seed)
    assert np.array_equal(r.fy, -r.fx)


@pytest.mark.parametrize("gpu_done", [True, False])
def test_rounds_advance_every_solve_by_min_remaining_round(monkeypatch, gpu_done):
    ws = [workload("a", 40, 10, 1200, 1), workload("b", 30, 10, 500, 2),
          workload("c", 20, 10, 900, 3)]
    reqs = [I.Request(i, 0.0, w) for i, w in enumerate(ws)]
    lib, srv, res, rep = serve(monkeypatch, reqs, 10**9, gpu_done, round_steps=500)
    assert lib.rounds == [[("a", 500), ("b", 500), ("c", 500)], [("a", 500), ("c", 400)],
                          [("a", 200)]]
    for w in ws:
        _check_series(res[w.name], w)
        assert res[w.name].error is None
    assert rep["completed"] == 3 and rep["failed"] == 0 and not srv.rejected
    assert rep["mlups"] > 0  # the figures themselves: test_report_percentiles
    assert lib.live_bytes == 0


@pytest.mark.parametrize("gpu_done", [True, False])
def test_fifo_admission_within_the_memory_budget(monkeypatch, gpu_done):
    """Two of the three large solves fit the budget: the third (c) waits
    until memory is released, and the small request d behind it waits too
    although it would fit beside a and b (first come, first served). The
    budget is never exceeded."""
    ws = [workload("a", 100, 10, 500, 1), workload("b", 100, 10, 1000, 2),
          workload("c", 100, 10, 500, 3), workload("d", 10, 10, 500, 4)]
    reqs = [I.Request(i, 0.0, w) for i, w in enumerate(ws)]
    budget = (2 * 100 * 10 + 10 * 10) * BYTES_PER_NODE  # a + b + d fit; c does not beside a, b
    lib, srv, res, rep = serve(monkeypatch, reqs, budget, gpu_done, round_steps=500)
    assert lib.peak_bytes <= budget
    assert lib.created == ["a", "b", "c", "d"]
    assert [n for n, _ in lib.rounds[0]] == ["a", "b"]
    assert all(res[w.name].admitted <= res[v.name].admitted for w, v in zip(ws, ws[1:]))
    for w in ws:
        _check_series(res[w.name], w)
    assert rep["completed"] == 4 and lib.live_bytes == 0


def test_slot_limit(monkeypatch):
    ws = [workload(n, 8, 8, 300 * (k + 1), k) for k, n in enumerate("abcde")]
    reqs = [I.Request(i, 0.0, w) for i, w in enumerate(ws)]
    lib, srv, res, rep = serve(monkeypatch, reqs, 10**9, True, max_active=2, round_steps=200)
    assert max(len(r) for r in lib.rounds) == 2
    assert sorted(res) == list("abcde")
    for w in ws:
        _check_series(res[w.name], w)


def test_requests_that_cannot_fit_or_be_created_are_refused_alone(monkeypatch):
    ws = [workload("big", 1000, 1000, 100, 1), workload("ok1", 10, 10, 300, 2),
          workload("broken", 10, 10, 300, 3), workload("ok2", 10, 10, 300, 4)]
    reqs = [I.Request(i, 0.0, w) for i, w in enumerate(ws)]
    lib, srv, res, rep = serve(monkeypatch, reqs, 10**6, True, round_steps=100,
                               fail_create=["broken"])
    assert srv.rejected == [0, 2]
    assert "out of device memory" in srv.errors[2]
    assert "big" not in lib.created and sorted(res) == ["ok1", "ok2"]
    for name in ("ok1", "ok2"):
        assert res[name].error is None


def test_a_diverging_solve_fails_alone(monkeypatch):
    ws = [workload("good", 10, 10, 400, 1), workload("bad", 10, 10, 400, 2),
          workload("late", 10, 10, 700, 3)]
    reqs = [I.Request(i, 0.0, w) for i, w in enumerate(ws)]
    lib, srv, res, rep = serve(monkeypatch, reqs, 10**6, False, round_steps=300,
                               diverge=["bad"])
    assert "diverged" in res["bad"].error
    assert res["good"].error is None and res["late"].error is None
    assert rep["failed"] == 1 and rep["completed"] == 3


def test_realtime_arrivals_are_admitted_after_they_arrive(monkeypatch):
    ws = [workload("now", 10, 10, 200, 1), workload("later", 10, 10, 200, 2)]
    reqs = [I.Request(0, 0.0, ws[0]), I.Request(1, 0.05, ws[1])]
    lib, srv, res, rep = serve(monkeypatch, reqs, 10**6, True, realtime=True, round_steps=100)
    assert res["later"].admitted >= 0.05
    assert res["later"].arrival == 0.05 and res["later"].latency == pytest.approx(
        res["later"].finished - 0.05)


def test_report_percentiles():
    lat = np.linspace(0.1, 10.0, 100)
    results = [S.Result(i, "r", 0.0, 0.0, float(x), 1000, 100_000, "f32", "srt")
               for i, x in enumerate(lat)]
    rep = S.Server.report(results, 20.0)
    assert rep["p50_latency_s"] == pytest.approx(np.percentile(lat, 50), abs=1e-4)
    assert rep["p99_latency_s"] == pytest.approx(np.percentile(lat, 99), abs=1e-4)
    assert rep["solves_per_s"] == 5.0
    assert rep["mlups"] == 100 * 1000 * 100_000 / 20.0 / 1e6  # 500 MLUPS


def test_report_counts_only_served_solves():
    """A failed solve (diverged or stopped) is neither served throughput nor a
    latency sample; its GPU work shows in mlups_all only."""
    lat = np.linspace(0.1, 10.0, 100)
    results = [S.Result(i, "r", 0.0, 0.0, float(x), 1000, 100_000, "f32", "srt",
                        error="diverged" if i % 4 == 0 else None) for i, x in enumerate(lat)]
    rep = S.Server.report(results, 20.0)
    ok = lat[np.arange(100) % 4 != 0]
    assert rep["completed"] == 100 and rep["served"] == 75 and rep["failed"] == 25
    assert rep["solves_per_s"] == 75 / 20.0
    assert rep["p50_latency_s"] == pytest.approx(np.percentile(ok, 50), abs=1e-4)
    assert rep["p99_latency_s"] == pytest.approx(np.percentile(ok, 99), abs=1e-4)
    assert rep["mlups"] == 75 * 1000 * 100_000 / 20.0 / 1e6
    assert rep["mlups_all"] == 100 * 1000 * 100_000 / 20.0 / 1e6


def test_deadlines_drop_waiting_requests_and_stop_running_ones(monkeypatch):
    """Fake clock, 1 ms per grouped step. "long" runs 3 rounds of 100 steps
    (0.3 s); "late" waits behind it for memory and its 0.15 s deadline passes
    first: dropped. "short" (deadline 0.15 s) is stopped at the first round
    boundary past it, with the force series of the steps it ran."""
    ws = [workload("long", 100, 10, 300, 1), workload("short", 10, 10, 400, 2),
          workload("late", 100, 10, 100, 3)]
    reqs = [I.Request(0, 0.0, ws[0]), I.Request(1, 0.0, ws[1], deadline=0.15),
            I.Request(2, 0.0, ws[2], deadline=0.15)]
    budget = (100 * 10 + 10 * 10) * BYTES_PER_NODE  # "late" cannot join "long"
    lib, srv, res, rep = serve(monkeypatch, reqs, budget, True, round_steps=100,
                               fake_clock=True)
    assert srv.dropped == {2: "deadline"} and "late" not in lib.created
    assert res["long"].error is None and res["long"].steps == 300
    assert res["short"].error == "deadline: stopped after 200 of 400 steps"
    assert res["short"].steps == 200 and len(res["short"].fx) == 200
    assert np.array_equal(res["short"].fx, np.arange(200) + 2000.0)
    assert rep["dropped"] == 1 and rep["stopped"] == 1 and rep["failed"] == 1
    assert lib.live_bytes == 0


@pytest.mark.parametrize("gpu_done", [True, False])
def test_cancel_drops_a_waiting_request_and_stops_a_running_one(monkeypatch, gpu_done):
    """Cancelled from the admission hook of "b" (any thread may call cancel):
    "a", admitted in the same pass, runs the round that follows and stops at
    the next round boundary; the waiting "c" is dropped when it reaches the
    head of the queue."""
    ws = [workload("a", 10, 10, 500, 1), workload("b", 10, 10, 300, 2),
          workload("c", 10, 10, 100, 3)]
    reqs = [I.Request(i, 0.0, w) for i, w in enumerate(ws)]
    srv_ref = {}

    def on_admit(req, solver):
        if req.rid == 1:
            srv_ref["srv"].cancel(0)
            srv_ref["srv"].cancel(2)

    lib = FakeLib()
    monkeypatch.setattr(S, "V", lib)
    srv = S.Server(10**6, stream=object(), round_steps=100, max_active=2, on_admit=on_admit)
    srv.torch = fake_torch(gpu_done)
    srv_ref["srv"] = srv
    results, rep = srv.run(reqs, realtime=False)
    res = {r.name: r for r in results}
    assert res["a"].error == "cancelled: stopped after 100 of 500 steps" and res["a"].steps == 100
    assert len(res["a"].fx) == 100
    assert res["b"].error is None and res["b"].steps == 300
    assert srv.dropped == {2: "cancelled"} and "c" not in lib.created
    assert rep["stopped"] == 1 and rep["dropped"] == 1


def test_one_log_line_per_request(monkeypatch):
    import io
    import json
    ws = [workload("big", 1000, 1000, 100, 1), workload("ok", 10, 10, 200, 2),
          workload("broken", 10, 10, 200, 3), workload("gone", 10, 10, 200, 4)]
    reqs = [I.Request(i, 0.0, w) for i, w in enumerate(ws)]
    reqs[3].deadline = -1.0  # already past: dropped at admission
    buf = io.StringIO()
    lib, srv, res, rep = serve(monkeypatch, reqs, 10**6, True, round_steps=100, log=buf,
                               fail_create=["broken"])
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    by = {x["rid"]: x for x in lines}
    assert len(lines) == 4 and sorted(by) == [0, 1, 2, 3]
    assert "over the budget" in by[0]["rejected"]
    assert by[1]["steps"] == 200 and by[1]["error"] is None and by[1]["nodes"] == 100
    assert by[1]["latency"] == pytest.approx(by[1]["finished"] - by[1]["arrival"])
    assert "out of device memory" in by[2]["rejected"]
    assert by[3]["dropped"] == "deadline"

