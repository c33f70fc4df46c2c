"""Serving loop: (frequency, source set) requests arriving over time.

Every frequency has its own Solver (mesh, factors and coarse factors stay
resident on the device) and its own hz_server with a fixed number of
right-hand-side slots. Admission is by free slots, which bound the device
footprint: the workspace of every frequency is allocated once, when its
server is created, and `hz_info.device_bytes` gives the total. Requests that
arrive while others are being solved join the shared block at the next
restart boundary (continuous batching); every server step runs one FGMRES
restart cycle for all the slots it holds. The loop reports per-request
latency (arrival to completion) and the throughput in right-hand sides per
second.
"""
from __future__ import annotations

import time

import numpy as np

from . import hz


class ServingLoop:
    def __init__(self, solvers, slots):
        """solvers: {frequency: hz.Solver}; slots: columns per frequency."""
        self.solvers = solvers
        self.servers = {f: hz.Server(S, slots) for f, S in solvers.items()}
        self.inflight = {}   # id -> (frequency, ns, arrival time)
        self.results = {}    # id -> (wavefields, stats, latency)

    def submit(self, request_id, freq, src_xyz, src_amp=None, arrival=None):
        self.servers[freq].submit(request_id, src_xyz, src_amp)
        self.inflight[request_id] = (freq, len(np.asarray(src_xyz).reshape(-1, 3)),
                                     time.perf_counter() if arrival is None else arrival)

    def busy(self):
        return any(sum(v.pending()) for v in self.servers.values())

    def step(self):
        """One restart cycle on every server that has work; returns the ids
        of the requests completed in this step."""
        done = []
        for v in self.servers.values():
            if sum(v.pending()) == 0:
                continue
            for rid in v.step():
                _, ns, t0 = self.inflight.pop(rid)
                u, st = v.fetch(rid, ns)
                self.results[rid] = (u, st, time.perf_counter() - t0)
                done.append(rid)
        return done

    def run_stream(self, requests, keep_wavefields=False):
        """requests: list of (arrival offset in s, id, frequency, src_xyz);
        submits each one when the wall clock reaches its arrival time and
        steps until every request has finished. Returns a summary."""
        order = sorted(requests, key=lambda r: r[0])
        t_start = time.perf_counter()
        i = 0
        while i < len(order) or self.busy():
            now = time.perf_counter() - t_start
            while i < len(order) and order[i][0] <= now:
                off, rid, f, src = order[i]
                self.submit(rid, f, src, arrival=t_start + off)
                i += 1
            if self.busy():
                for rid in self.step():
                    if not keep_wavefields:
                        u, st, lat = self.results[rid]
                        self.results[rid] = (None, st, lat)
            elif i < len(order):
                time.sleep(min(0.01, max(0.0, order[i][0] - now)))
        wall = time.perf_counter() - t_start
        lat = np.array([self.results[r[1]][2] for r in order])
        nrhs = sum(len(np.asarray(r[3]).reshape(-1, 3)) for r in order)
        return {"requests": len(order), "rhs": int(nrhs), "wall_s": wall, "rhs_per_s": nrhs / wall,
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "converged": all(self.results[r[1]][1]["converged"] for r in order)}

    def close(self):
        for v in self.servers.values():
            v.close()
