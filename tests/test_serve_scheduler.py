"""Host logic of the serving loop (paper_2505_12958_gb300.serve.Server) on the CPU.

The device side (contexts, streams, events) is replaced by fakes that record what the server
asks for, so these tests check the scheduling rules alone: first-come-first-served admission
without overtaking while the summed footprints fit the memory budget (a request larger than
the budget runs alone), the cap on active requests, chunks of at most `chunk` steps that add
up to each request's step count, refusal at admission without holding budget, retirement of
every request exactly once, and the batched form's split between one batch call for the small
requests and per-context steps for the large ones.
"""
import time
import types

import numpy as np
import pytest

serve = pytest.importorskip("paper_2505_12958_gb300.serve")


class FakeError(Exception):
    pass


class World:
    """Fake device: contexts count their steps; an event completes `lag` queries after it is
    recorded; the budget ledger is checked on every admission."""

    def __init__(self, lag=1, fail_ids=()):
        self.lag = lag
        self.fail_ids = set(fail_ids)
        self.live = {}            # request id -> fake context
        self.trace = []           # ("admit" | "step" | "batch" | "close", id, k)
        self.max_live = 0

    def context(self, owner):
        world = self

        class Ctx:
            def __init__(self, eam, ace, box, x, v, fixed, region, indenter, ind_vel, mass, precision=None,
                         stream=None, list_sizing=None):
                rid = int(box["id"])
                if rid in world.fail_ids:
                    raise FakeError("AP_ERR_OOM: injected")
                self.rid, self.n, self.steps, self.closed = rid, len(x), 0, False
                world.live[rid] = self
                world.max_live = max(world.max_live, len(world.live))
                world.trace.append(("admit", rid, 0))
                owner.check_budget()

            def step(self, k, dt):
                assert not self.closed
                self.steps += k
                world.trace.append(("step", self.rid, k))

            def energy(self):
                return {"n_ace": 0, "e_total": float(self.steps)}

            def get_state(self):
                return np.zeros((self.n, 3)), np.zeros((self.n, 3)), 0.0

            def forces(self):
                return np.zeros((self.n, 3), dtype=np.float32)

            def memory_bytes(self):
                return 1

            def close(self):
                self.closed = True
                del world.live[self.rid]
                world.trace.append(("close", self.rid, self.steps))

        return Ctx

    def torch(self):
        world = self

        class Event:
            def __init__(self):
                self.left = None

            def record(self, stream):
                self.left = world.lag

            def query(self):
                if self.left > 0:
                    self.left -= 1
                    return False
                return True

        cuda = types.SimpleNamespace(Stream=lambda: object(), Event=Event, mem_get_info=lambda: (1 << 40, 1 << 40))
        return types.SimpleNamespace(cuda=cuda)


def make_requests(sizes, steps, arrivals=None):
    reqs = []
    for k, (n, s) in enumerate(zip(sizes, steps)):
        reqs.append({"id": k, "x": np.zeros((n, 3)), "v": None, "fixed": None, "box": {"id": k}, "region": None,
                     "eam": None, "ace": None, "mass": 1.0, "n_steps": s,
                     "arrival_s": 0.0 if arrivals is None else arrivals[k]})
    return reqs


def run_server(monkeypatch, reqs, feet, world, **kw):
    monkeypatch.setattr(serve, "APError", FakeError)
    monkeypatch.setattr(serve, "torch", world.torch())
    by_n = {}

    def footprint(eam, ace, n, mass):
        return by_n[n]

    batches = []

    def step_batch(ctxs, ks, dt, stream):
        batches.append([(c.rid, k) for c, k in zip(ctxs, ks)])
        for c, k in zip(ctxs, ks):
            c.steps += k
            world.trace.append(("batch", c.rid, k))

    monkeypatch.setattr(serve, "footprint_bytes", footprint)
    monkeypatch.setattr(serve, "step_batch", step_batch)
    for r, f in zip(reqs, feet):
        assert by_n.get(len(r["x"]), f) == f          # footprint is a function of the size here
        by_n[len(r["x"])] = f
    srv = serve.Server(**kw)
    world.check_budget = lambda: None
    monkeypatch.setattr(serve, "APContext", world.context(world))
    done = srv.run(reqs, realtime=False)
    # replay the trace: at every admission the live footprints fit the budget, or the new
    # request runs alone
    live = set()
    for kind, rid, _ in world.trace:
        if kind == "admit":
            live.add(rid)
            assert sum(feet[q] for q in live) <= srv.mem_budget or live == {rid}, (rid, live)
        elif kind == "close":
            live.discard(rid)
    return srv, done, batches


def test_every_request_completes_once_with_all_its_steps(monkeypatch):
    rng = np.random.default_rng(1)
    sizes = [int(s) for s in rng.integers(10, 500, 40)]
    steps = [int(s) for s in rng.integers(1, 30, 40)]
    world = World(lag=2)
    srv, done, _ = run_server(monkeypatch, make_requests(sizes, steps), sizes, world, mem_budget=10**9, chunk=8,
                              max_active=7)
    assert sorted(r.id for r in done) == list(range(40))
    assert all(r.error is None for r in done)
    for r in done:
        assert r.energy["e_total"] == steps[r.id]
        assert r.done_s >= r.admit_s >= r.arrival_s
    chunks = [(rid, k) for kind, rid, k in world.trace if kind == "step"]
    for rid in range(40):
        ks = [k for q, k in chunks if q == rid]
        assert sum(ks) == steps[rid] and max(ks) <= 8
    assert world.max_live <= 7 and srv.peak_active <= 7
    assert srv.used == 0 and not world.live


def test_admission_is_fifo_within_the_memory_budget(monkeypatch):
    # footprints 60, 50, 30, 20 with budget 100: the 50 must wait for the 60 to leave although
    # the 30 behind it would fit (no overtaking); a request above the budget runs alone
    sizes = [60, 50, 30, 20, 150, 10]
    steps = [16, 8, 8, 8, 8, 8]
    world = World(lag=1)
    t0 = time.perf_counter()
    srv, done, _ = run_server(monkeypatch, make_requests(sizes, steps), sizes, world, mem_budget=100, chunk=8)
    # whenever every active request retires while the queue waits (here after requests 0, 3
    # and 4), the next request is admitted in the next pass, without idling
    assert time.perf_counter() - t0 < 0.5
    admits = [rid for kind, rid, _ in world.trace if kind == "admit"]
    assert admits == list(range(6))
    order = [(kind, rid) for kind, rid, _ in world.trace if kind in ("admit", "close")]
    assert order.index(("close", 0)) < order.index(("admit", 1))
    big = order.index(("admit", 4))
    assert all(("close", q) in order[:big] for q in range(4))
    assert order.index(("close", 4)) < order.index(("admit", 5))
    assert srv.peak_used == 150 and srv.used == 0


def test_refused_request_holds_no_budget_and_the_others_finish(monkeypatch):
    sizes = [40, 41, 42, 43]
    steps = [5, 5, 5, 5]
    world = World(lag=0, fail_ids={1})
    srv, done, _ = run_server(monkeypatch, make_requests(sizes, steps), sizes, world, mem_budget=10**6)
    by_id = {r.id: r for r in done}
    assert sorted(by_id) == [0, 1, 2, 3]
    assert "AP_ERR_OOM" in by_id[1].error and by_id[1].energy is None and by_id[1].footprint_bytes == 41
    assert all(by_id[k].error is None and by_id[k].energy["e_total"] == 5 for k in (0, 2, 3))
    assert srv.used == 0


def test_batched_form_sends_small_requests_through_one_call(monkeypatch):
    sizes = [100, 2000, 300, 5000, 50]
    steps = [12, 12, 12, 12, 12]
    world = World(lag=1)
    srv, done, batches = run_server(monkeypatch, make_requests(sizes, steps), sizes, world, mem_budget=10**9,
                                    chunk=8, batched=True, batch_atoms=1024)
    assert sorted(r.id for r in done) == list(range(5))
    small, big = {0, 2, 4}, {1, 3}
    assert batches and all({rid for rid, _ in b} <= small for b in batches)
    assert {rid for kind, rid, _ in world.trace if kind == "step"} == big
    for rid in range(5):
        assert sum(k for kind, q, k in world.trace if q == rid and kind in ("step", "batch")) == 12
