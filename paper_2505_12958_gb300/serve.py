"""Serving form: many independent structures stepped concurrently on one GPU.

Continuous batching over whole MD requests.  Each admitted request gets its own context
(`APContext`) on its own non-blocking stream, with its neighbour list sized from the density
bound, so that creating it never waits for the GPU.  In every scheduling pass the server issues
one chunk of velocity-Verlet steps for every active request: by default each request
replays its own step graphs on its own stream, so the requests' kernels overlap on the
device; with `batched`, the requests of at most `batch_atoms` atoms go through one
`ap_step_batch` call on the server's stream instead, where every stage of a step is one
kernel launch for all of them (per-atom stages give each request its own blocks, the ACE
stages share one persistent grid over the compacted atoms of all requests).  Requests
join at any pass once their device footprint (`ap_footprint_bytes`) fits the memory budget
(first come, first served, no overtaking) and leave as soon as their last chunk has
completed, which the server learns from a CUDA event without blocking the others.

Latency runs from a request's arrival to the moment its final positions, velocities,
forces and energy are readable on the host.  A request's results do not depend on what it
is batched with: every kernel is deterministic and contexts share no device state.

A request that fails is reported in its Result (`error`, the library status text) and
leaves the others untouched: one whose context cannot be created (for instance AP_ERR_OOM)
is refused at admission, one whose steps end in a device error (AP_ERR_DOMAIN,
AP_ERR_LIMIT, ...) is retired with that error when it completes.
"""
import collections
import time

import numpy as np
import torch

from . import APContext, APError, footprint_bytes, step_batch

__all__ = ["Server", "Result", "percentile_ms"]


class Result:
    __slots__ = ("id", "n_atoms", "n_steps", "n_ace", "arrival_s", "admit_s", "done_s", "energy",
                 "x", "v", "forces", "memory_bytes", "footprint_bytes", "error")

    @property
    def latency_s(self):
        return self.done_s - self.arrival_s


class _Active:
    __slots__ = ("req", "ctx", "stream", "left", "events", "foot", "admit_s")


class Server:
    """Continuous-batching MD server on the current CUDA device.

    mem_budget   device bytes the active contexts may hold (default: 80 % of free memory)
    chunk        MD steps issued per request per scheduling pass
    max_active   cap on concurrently active requests
    inflight     chunks a request may have queued on its stream at once
    keep_arrays  keep final x, v, forces in each Result (else only the energy report)
    batched      one ap_step_batch call per pass for the requests of at most batch_atoms
                 atoms (every stage one launch for all of them); larger requests, which fill
                 the GPU by themselves, step with their own replayed graphs on their own
                 streams beside the batch.  False (the default, lower latency) steps every
                 request on its own stream.
    """

    def __init__(self, mem_budget=None, chunk=8, dt=1.0, max_active=64, inflight=2, precision="fp32",
                 keep_arrays=True, batched=False, batch_atoms=1024):
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info()
            mem_budget = int(0.8 * free)
        self.mem_budget = int(mem_budget)
        self.chunk = int(chunk)
        self.dt = float(dt)
        self.max_active = int(max_active)
        self.inflight = int(inflight)
        self.precision = precision
        self.keep_arrays = keep_arrays
        self.batched = batched
        self.batch_atoms = int(batch_atoms)
        self._streams = []
        self.stream = torch.cuda.Stream()       # the batched launches
        self.used = 0
        self.peak_used = 0
        self.peak_active = 0
        self.passes = 0

    def _stream(self):
        return self._streams.pop() if self._streams else torch.cuda.Stream()

    @staticmethod
    def _failed(req, now, err, foot=0):
        r = Result()
        r.id, r.n_atoms, r.n_steps = req["id"], len(req["x"]), int(req["n_steps"])
        r.arrival_s, r.admit_s, r.done_s = req["arrival_s"], now, now
        r.energy, r.n_ace = None, 0
        r.x = r.v = r.forces = None
        r.memory_bytes, r.footprint_bytes = 0, foot
        r.error = str(err)
        return r

    def _admit(self, req, foot, now):
        """The request's context on its own stream, or (None, refused Result) when it cannot
        be created."""
        a = _Active()
        a.req, a.foot, a.admit_s = req, foot, now
        a.stream = self._stream()
        try:
            a.ctx = APContext(req["eam"], req["ace"], req["box"], req["x"], req["v"], req["fixed"], req["region"],
                              req.get("indenter"), req.get("ind_vel"), req["mass"], precision=self.precision,
                              stream=a.stream, list_sizing="bound")
        except APError as e:
            self._streams.append(a.stream)
            return None, self._failed(req, now, e, foot)
        a.left = int(req["n_steps"])
        a.events = collections.deque()
        self.used += foot
        self.peak_used = max(self.peak_used, self.used)
        return a, None

    def _retire(self, a, t0):
        r = Result()
        q = a.req
        r.id, r.n_atoms, r.n_steps = q["id"], len(q["x"]), int(q["n_steps"])
        r.arrival_s, r.admit_s = q["arrival_s"], a.admit_s
        r.error = None
        r.x = r.v = r.forces = None
        try:
            r.energy = a.ctx.energy()
            r.n_ace = r.energy["n_ace"]
            if self.keep_arrays:
                r.x, r.v, _ = a.ctx.get_state()
                r.forces = a.ctx.forces()
        except APError as e:
            r.energy, r.n_ace, r.error = None, 0, str(e)
        r.memory_bytes = a.ctx.memory_bytes()
        r.footprint_bytes = a.foot
        r.done_s = time.perf_counter() - t0
        a.ctx.close()
        self._streams.append(a.stream)
        self.used -= a.foot
        return r

    def run(self, requests, realtime=True):
        """Serve `requests` (dicts with x, v, box, ..., n_steps, arrival_s).  With realtime,
        request k becomes visible at its arrival_s after the start; otherwise all are
        visible at once (closed loop, for the saturated throughput).  Returns the Results in
        completion order."""
        reqs = sorted(requests, key=lambda r: r["arrival_s"])
        if not realtime:
            reqs = [dict(r, arrival_s=0.0) for r in reqs]
        feet = [footprint_bytes(r["eam"], r["ace"], len(r["x"]), r["mass"]) for r in reqs]
        k_next = 0
        queue = collections.deque()
        active = []
        done = []
        t0 = time.perf_counter()
        while k_next < len(reqs) or queue or active:
            now = time.perf_counter() - t0
            while k_next < len(reqs) and reqs[k_next]["arrival_s"] <= now:
                queue.append((reqs[k_next], feet[k_next]))
                k_next += 1
            # admission: first come, first served while the footprint fits
            while queue and len(active) < self.max_active:
                q, foot = queue[0]
                if active and self.used + foot > self.mem_budget:
                    break
                queue.popleft()
                a, refused = self._admit(q, foot, time.perf_counter() - t0)
                if a is None:
                    done.append(refused)
                else:
                    active.append(a)
            self.peak_active = max(self.peak_active, len(active))
            # retire finished requests; trim completed chunk events
            still = []
            for a in active:
                while a.events and a.events[0].query():
                    a.events.popleft()
                if a.left == 0 and not a.events:
                    done.append(self._retire(a, t0))
                else:
                    still.append(a)
            active = still
            # one chunk for every request with room in its stream queue
            batch = [a for a in active if a.left > 0 and len(a.events) < self.inflight]
            if batch:
                ks = [min(self.chunk, a.left) for a in batch]
                try:
                    small = [q for q, a in enumerate(batch) if self.batched and len(a.req["x"]) <= self.batch_atoms]
                    if small:
                        step_batch([batch[q].ctx for q in small], [ks[q] for q in small], self.dt, self.stream)
                    big = set(range(len(batch))) - set(small)
                    for q in sorted(big):
                        batch[q].ctx.step(ks[q], self.dt)
                except APError:
                    # a launch was refused: every context was still issued; the failing ones
                    # report their status when they retire
                    pass
                for a, k in zip(batch, ks):
                    a.left -= k
                    ev = torch.cuda.Event()
                    ev.record(a.stream)
                    a.events.append(ev)
                self.passes += 1
            elif not active and (queue or k_next == len(reqs)):
                # every active request retired in this pass: admit the head of the queue now
                # (it waited for room) instead of idling until the next arrival, or end the
                # run when nothing is left to arrive
                continue
            else:
                # nothing to issue: wait for a completion or the next arrival
                nxt = reqs[k_next]["arrival_s"] - (time.perf_counter() - t0) if k_next < len(reqs) else 1.0
                time.sleep(min(max(nxt, 0.0), 5e-5) if active else max(nxt, 0.0))
        return done


def percentile_ms(results, q):
    lat = np.array([r.latency_s for r in results]) * 1e3
    return float(np.percentile(lat, q)) if len(lat) else float("nan")
