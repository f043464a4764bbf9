"""Serving: continuous batching over grouped launches. Each solve's result is
the same alone and in the mix (bitwise: the grouped kernel is the single-solver
kernel with deterministic reductions), admission respects the memory budget,
and requests arriving while others run are admitted and finish."""
import numpy as np
import pytest

from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1812_05401_gb300 import build as B
    B.build()
    from paper_1812_05401_gb300 import serve, vplbm
    return serve, vplbm


def _small_mix(n=14, seed=7):
    reqs = I.serving_mix(n, rate=400.0, seed=seed, side_min=24, side_max=96, steps_min=40,
                         steps_max=260)
    return reqs


def test_results_identical_alone_and_in_the_mix(mods):
    serve, V = mods
    reqs = _small_mix()
    srv = serve.Server(budget_bytes=1 << 30, max_active=6, round_steps=64, keep_populations=True)
    results, rep = srv.run(reqs, realtime=False)
    assert rep["completed"] == len(reqs) and not srv.rejected
    by_id = {r.rid: r for r in results}
    for req in reqs[::3]:
        with V.Solver.from_workload(req.workload, ring_len=max(1, req.workload.steps),
                                    reduce_mass=False, tile_rows=serve.SERVE_TILE_ROWS) as s:
            s.step(req.workload.steps)
            f = s.populations()
            fx, fy, _ = s.forces()
        r = by_id[req.rid]
        assert np.array_equal(f, r.populations), req.workload.name
        assert np.array_equal(fx, r.fx) and np.array_equal(fy, r.fy)


def test_admission_by_memory_budget(mods):
    serve, V = mods
    reqs = _small_mix(8, seed=11)
    fps = []
    for r in reqs:
        cfg, _ = V.config_from_workload(r.workload, ring_len=max(1, r.workload.steps),
                                        tile_rows=serve.SERVE_TILE_ROWS)
        fps.append(V.vplbm_footprint_bytes(cfg))
    budget = max(fps) + min(fps)  # at most about two solves at a time
    srv = serve.Server(budget_bytes=budget, max_active=8, round_steps=32)
    results, rep = srv.run(reqs, realtime=False)
    assert rep["completed"] == len(reqs)
    # a request larger than the whole budget is rejected, not served
    big = I.serving_mix(1, seed=3, side_min=900, side_max=1000, steps_min=10, steps_max=10)
    srv2 = serve.Server(budget_bytes=budget, max_active=8, round_steps=32)
    res2, rep2 = srv2.run(big, realtime=False)
    assert rep2["completed"] == 0 and srv2.rejected == [big[0].rid]


def test_late_arrivals_join_running_rounds(mods):
    serve, V = mods
    reqs = I.serving_mix(10, rate=400.0, seed=5, side_min=24, side_max=64, steps_min=1500,
                         steps_max=3000)
    # spread arrivals so that later ones arrive while earlier ones run
    for i, r in enumerate(reqs):
        r.arrival = 0.003 * i
    srv = serve.Server(budget_bytes=1 << 30, max_active=8, round_steps=100)
    results, rep = srv.run(reqs, realtime=True)
    assert rep["completed"] == len(reqs)
    assert all(r.finished >= r.arrival for r in results)
    overlapped = sum(1 for a in results for b in results
                     if a.rid != b.rid and a.admitted < b.finished and b.admitted < a.finished)
    assert overlapped > 0
    assert rep["p99_latency_s"] >= rep["p50_latency_s"] > 0


def test_a_diverging_solve_fails_alone(mods):
    """Failure isolation: one request is given a non-finite state (written from
    the host right after admission); it is reported as diverged and every other
    request in the same grouped launches completes with the result it has alone."""
    serve, V = mods
    import numpy as np
    reqs = _small_mix(8, seed=21)
    bad = reqs[3].rid

    def poison(req, solver):
        if req.rid == bad:
            f = solver.populations()
            f[:, 2, 2] = np.nan
            solver.set_populations(f)

    srv = serve.Server(budget_bytes=1 << 30, max_active=8, round_steps=32, keep_populations=True,
                       on_admit=poison)
    results, rep = srv.run(reqs, realtime=False)
    assert rep["completed"] == len(reqs) and rep["failed"] == 1
    by_id = {r.rid: r for r in results}
    assert by_id[bad].error and "diverged" in by_id[bad].error
    for req in reqs:
        if req.rid == bad:
            continue
        assert by_id[req.rid].error is None
        with V.Solver.from_workload(req.workload, ring_len=max(1, req.workload.steps),
                                    reduce_mass=False, device_init=True,
                                    tile_rows=serve.SERVE_TILE_ROWS) as s:
            s.step(req.workload.steps)
            assert np.array_equal(s.populations(), by_id[req.rid].populations)


def test_fp16_store_serves_steady_drag_within_1e3_of_fp32(mods):
    """The serving precision bar: the same requests served with FP16-offset
    storage and with FP32 storage give mean drag coefficients (second half of
    the run) within 1e-3 of each other where the drag is stationary: cylinder
    channels below the onset of vortex shedding (Re < 47), SRT and MRT, of
    the mix's smaller sizes, 20,000 steps each. Every solve succeeds."""
    serve, V = mods
    from paper_1812_05401_gb300 import diag
    reqs = {"f32": [], "f16": []}
    rid = 0
    for side in (64, 96, 128):
        for re in (25.0, 40.0):
            d = max(4.0, round(40.0 * side / 256.0))
            for st in reqs:
                w = I.cylinder_channel(4 * side, side, d, 0.05, re, 20_000,
                                       collision="srt" if rid % 2 else "mrt", storage=st,
                                       perturbation=1e-4, seed=100 + rid)
                reqs[st].append(I.Request(rid, 0.0, w))
            rid += 1
    served = {}
    for st, rq in reqs.items():
        srv = serve.Server(budget_bytes=1 << 32, max_active=16, round_steps=500)
        results, rep = srv.run(rq, realtime=False)
        assert rep["failed"] == 0 and rep["served"] == len(rq)
        served[st] = {r.rid: r for r in results}
    for req in reqs["f32"]:
        w = req.workload
        cd = []
        for st in ("f32", "f16"):
            r = served[st][req.rid]
            c, _ = diag.coefficients(r.fx, r.fy, w.u_ref, w.l_ref)
            cd.append(float(np.mean(c[len(c) // 2:])))
        rel = abs(cd[1] - cd[0]) / abs(cd[0])
        print(w.name, w.collision, "C_D f32", cd[0], "f16", cd[1], "rel", rel)
        assert rel < 1e-3, w.name
