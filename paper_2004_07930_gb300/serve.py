"""Serving loop: (frequency, source set) requests arriving over time.

Every frequency has its own Solver (mesh, factors and coarse factors stay
resident on the device) and its own hz_server. Admission is by device
footprint: a server's slot count is its share of the device budget divided by
the bytes one right-hand-side column costs on that solver
(hz_server_column_bytes: the column's share of the Krylov basis, the
preconditioner blocks and the local sub-vectors), and a request's sources
wait in the server's queue until slots (and so the memory reserved for them)
free up. The workspace is allocated once, when a server is created, so
admission never allocates. Requests that arrive while others are being
solved join the shared block at the next restart boundary (continuous
batching). Each frequency's server is stepped by its own host thread, so the
device work of different frequencies overlaps (every context has its own
stream). The loop reports per-request latency (arrival to completion) and the
throughput in right-hand sides per second.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import hz


def slots_for_budget(solvers, device_budget, max_slots=64):
    """Slots per frequency: an equal share of `device_budget` bytes divided by
    the bytes of one column on that frequency's solver, rounded down to a
    power of two (the kernels run the instantiation for the next power of two
    of the block width, so other widths pay for idle columns), at least 1."""
    share = float(device_budget) / len(solvers)
    out = {}
    for f, S in solvers.items():
        n = int(max(1, min(max_slots, share // S.column_bytes())))
        out[f] = 1 << (n.bit_length() - 1)
    return out


class ServingLoop:
    def __init__(self, solvers, slots=None, device_budget=None):
        """solvers: {frequency: hz.Solver}; slots: columns per frequency (int
        or {frequency: int}), or device_budget: bytes shared by the servers."""
        self.solvers = solvers
        if device_budget is not None:
            self.slots = slots_for_budget(solvers, device_budget)
        elif isinstance(slots, dict):
            self.slots = dict(slots)
        else:
            self.slots = {f: int(slots) for f in solvers}
        self.servers = {f: hz.Server(S, self.slots[f]) for f, S in solvers.items()}
        self.inflight = {}   # id -> (frequency, ns, arrival time)
        self.results = {}    # id -> (wavefields, stats, latency)
        self._lock = threading.Lock()
        self._incoming = {f: [] for f in solvers}   # submissions the frequency's worker has not taken yet
        self.errors = []

    def submit(self, request_id, freq, src_xyz, src_amp=None, arrival=None):
        """Queue a request (thread-safe); its server's worker submits it
        before the next step."""
        with self._lock:
            self.inflight[request_id] = (freq, len(np.asarray(src_xyz).reshape(-1, 3)),
                                         time.perf_counter() if arrival is None else arrival)
            self._incoming[freq].append((request_id, src_xyz, src_amp))

    def _take(self, f):
        with self._lock:
            new, self._incoming[f] = self._incoming[f], []
        for rid, src, amp in new:
            self.servers[f].submit(rid, src, amp)

    def busy(self, f=None):
        fs = [f] if f is not None else list(self.servers)
        with self._lock:
            if any(self._incoming[q] for q in fs):
                return True
        return any(sum(self.servers[q].pending()) for q in fs)

    def step(self, f):
        """One restart cycle on the server of frequency f (if it has work);
        returns the ids of the requests completed in this step."""
        self._take(f)
        v = self.servers[f]
        if sum(v.pending()) == 0:
            return []
        done = []
        for rid in v.step():
            with self._lock:
                _, ns, t0 = self.inflight.pop(rid)
            u, st = v.fetch(rid, ns)
            lat = time.perf_counter() - t0
            with self._lock:
                self.results[rid] = (u, st, lat)
            done.append(rid)
        return done

    def _worker(self, f, stop, keep_wavefields):
        try:
            while not stop.is_set() or self.busy(f):
                if self.busy(f):
                    for rid in self.step(f):
                        if not keep_wavefields:
                            with self._lock:
                                u, st, lat = self.results[rid]
                                self.results[rid] = (None, st, lat)
                else:
                    time.sleep(0.002)
        except Exception as e:  # reported by run_stream
            self.errors.append(e)

    def run_stream(self, requests, keep_wavefields=False):
        """requests: list of (arrival offset in s, id, frequency, src_xyz);
        submits each one when the wall clock reaches its arrival time while
        one worker thread per frequency steps its server, until every request
        has finished. Returns a summary."""
        order = sorted(requests, key=lambda r: r[0])
        stop = threading.Event()
        workers = [threading.Thread(target=self._worker, args=(f, stop, keep_wavefields), daemon=True)
                   for f in self.servers]
        t_start = time.perf_counter()
        for w in workers:
            w.start()
        for off, rid, f, src in order:
            now = time.perf_counter() - t_start
            if off > now:
                time.sleep(off - now)
            self.submit(rid, f, src, arrival=t_start + off)
        stop.set()
        for w in workers:
            w.join()
        if self.errors:
            raise self.errors[0]
        wall = time.perf_counter() - t_start
        lat = np.array([self.results[r[1]][2] for r in order])
        nrhs = sum(len(np.asarray(r[3]).reshape(-1, 3)) for r in order)
        return {"requests": len(order), "rhs": int(nrhs), "wall_s": wall, "rhs_per_s": nrhs / wall,
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "converged": all(self.results[r[1]][1]["converged"] for r in order),
                "slots": {str(f): n for f, n in self.slots.items()}}

    def close(self):
        for v in self.servers.values():
            v.close()
