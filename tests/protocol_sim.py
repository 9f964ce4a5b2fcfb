"""CPU-thread model of the asynchronous run's exchange protocol (test
infrastructure).

One Python thread per segment plays the CTA of the asynchronous kernel: at
step k it takes, for each neighbour, the newest published version v <= k of
that neighbour's facing edge value, waiting (with a time limit) only while
v < k-q+1 (Section 3, Eq. (eqn:async): k* in {k, ..., k-q+1}); it records
d = k - v, advances its own points one step, writes its two new edge values
into its ring slot (k+1) mod R and then publishes version k+1.  A replay
waits for exactly v = k - d.  The rings hold R >= 2q versions; every entry
carries the version it was written for, so a read of a slot that was already
overwritten (the race the ring length must rule out) is detected, as is a
read of a version newer than k.  A segment whose `stall` flag is set never
publishes: its neighbours' waits run out and every thread stops with the
status "timeout", as the kernel's bounded waits do.

Ring safety: publishing version k+1 overwrites the slot of version k+1-R.
The writer has read its neighbours' versions >= k-q+1, so each neighbour is
at a step k' >= k-q+1 and reads versions >= k'-q+1 >= k-2q+2 > k+1-R when
R >= 2q; the version tags check this on every read.

The state arithmetic is numpy's unfused r*((uR - 2u) + uL) + u; the model
checks the protocol, not the rounding (the oracle replays its traces to
within a few ulps).
"""
from __future__ import annotations

import random
import threading
import time

import numpy as np


class ProtocolError(AssertionError):
    pass


def segment_offsets(N, S):
    base, extra = divmod(N, S)
    off = [0]
    for s in range(S):
        off.append(off[-1] + base + (1 if s < extra else 0))
    return off


class AsyncProtocol:
    def __init__(self, u0, r, c1, cN, S, q, K, trace=None, stall=-1, limit_s=2.0, jitter_s=2e-4, seed=0):
        self.u = np.array(u0, dtype=np.float64)
        self.u[0], self.u[-1] = c1, cN
        self.N, self.r, self.S, self.q, self.K = len(self.u), float(r), int(S), int(q), int(K)
        self.R = 1
        while self.R < 2 * self.q:
            self.R *= 2
        self.off = segment_offsets(self.N, self.S)
        self.trace_in = None if trace is None else np.asarray(trace, dtype=np.uint8)
        self.trace = np.zeros((self.K, max(self.S - 1, 0), 2), dtype=np.uint8)
        self.stall = stall
        self.limit_s = limit_s
        self.jitter_s = jitter_s
        self.seed = seed
        # rings[s][side][slot] = (version, value); side 0: first point, 1: last point
        self.rings = [[[(-1, 0.0)] * self.R for _ in range(2)] for _ in range(self.S)]
        self.prog = [0] * self.S  # newest version published (version 0 = the initial state)
        self.lock = threading.Lock()  # stands for the release/acquire pairs of the kernel
        self.status = "ok"
        for s in range(self.S):
            lo, hi = self.off[s], self.off[s + 1]
            self.rings[s][0][0] = (0, self.u[lo])
            self.rings[s][1][0] = (0, self.u[hi - 1])
        self.max_lead = 0

    def _fail(self, what):
        with self.lock:
            if self.status == "ok":
                self.status = what

    def _read(self, s_nb, side, k, tidx, d_replay):
        """Newest (free) or recorded (replay) version of a neighbour's edge."""
        need = k - min(d_replay, k) if d_replay is not None else max(k - self.q + 1, 0)
        if d_replay is not None and d_replay >= self.q:
            self._fail("trace")
            return None
        t0 = time.monotonic()
        while True:
            with self.lock:
                V = self.prog[s_nb]
                if self.status != "ok":
                    return None
                if V >= need:
                    v = need if d_replay is not None else min(V, k)
                    ver, val = self.rings[s_nb][side][v % self.R]
                    if ver != v:
                        raise ProtocolError("segment read version %d from a slot holding version %d" % (v, ver))
                    if v > k:
                        raise ProtocolError("read a version newer than the step")
                    self.trace[k][tidx[0]][tidx[1]] = k - v
                    return val
            if time.monotonic() - t0 > self.limit_s:
                self._fail("timeout")
                return None
            time.sleep(0)

    def _segment(self, s):
        rng = random.Random(self.seed * 1000 + s)
        lo, hi = self.off[s], self.off[s + 1]
        x = self.u[max(lo - 1, 0):min(hi + 1, self.N)].copy()  # own points plus one halo point per side
        has_l, has_r = s > 0, s + 1 < self.S
        il = 1 if has_l else 0  # index of the first own point in x
        for k in range(self.K):
            if self.status != "ok":
                return
            if self.jitter_s:
                time.sleep(rng.random() * self.jitter_s)
            if has_l:
                d = None if self.trace_in is None else int(self.trace_in[k][s - 1][1])
                val = self._read(s - 1, 1, k, (s - 1, 1), d)
                if val is None:
                    return
                x[0] = val
            if has_r:
                d = None if self.trace_in is None else int(self.trace_in[k][s][0])
                val = self._read(s + 1, 0, k, (s, 0), d)
                if val is None:
                    return
                x[-1] = val
            y = x.copy()
            a, b = 1, len(x) - 1  # interior of x: every point with both neighbours in x
            y[a:b] = self.r * ((x[a + 1:b + 1] - 2.0 * x[a:b]) + x[a - 1:b - 1]) + x[a:b]
            if lo == 0:
                y[0] = self.u[0]  # the Dirichlet end u_1 (held)
            if hi == self.N:
                y[-1] = self.u[-1]
            x = y
            if s == self.stall:
                continue  # never publishes
            with self.lock:
                slot = (k + 1) % self.R
                self.rings[s][0][slot] = (k + 1, x[il])
                self.rings[s][1][slot] = (k + 1, x[il + (hi - lo) - 1])
                self.prog[s] = k + 1
                lead = max((k + 1) - self.prog[n] for n in (s - 1, s + 1) if 0 <= n < self.S) if self.S > 1 else 0
                self.max_lead = max(self.max_lead, lead)
        with self.lock:
            self.u[lo:hi] = x[il:il + (hi - lo)]

    def _segment_checked(self, s):
        try:
            self._segment(s)
        except ProtocolError as e:  # reported through the status, as the kernel's status word
            self._fail("protocol: %s" % e)

    def run(self):
        threads = [threading.Thread(target=self._segment_checked, args=(s,), daemon=True) for s in range(self.S)]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=self.limit_s * (self.K + 10))
        return self.status


class BlockedProtocol:
    """CPU-thread model of the blocked asynchronous run's exchange (strips of
    T edge points once per block of T steps) on segments given by S+1
    offsets: the on-chip blocked kernel's segments and the parts of a split
    rod in the batched launch.

    Segment s starts block b from a tile of its own points and T halo points
    per side (clipped at the rod's ends), the halos being the neighbours'
    strips of version v -- their first / last T points after v blocks.  In a
    free run v is the newest version published, not newer than b, waiting
    (with a time limit) only while v < b-q+1; a replay takes exactly
    v = b - d.  It sweeps the tile tb = min(T, K - bT) times (tile edges and
    Dirichlet ends held), keeps its own points, writes its first and last T
    points as strip version b+1 into ring slot (b+1) mod R and publishes the
    version.  The rings hold R >= 2q versions, every entry tagged with its
    version, so a read of an overwritten slot is detected.  Delays are
    recorded as trace[b][boundary][side], side 0 the left segment's read of
    its right neighbour, side 1 the right segment's read of its left one.
    The arithmetic is numpy's unfused one (the model checks the protocol, not
    the rounding).  periodic=True: the segments form a ring (Section 5.3):
    segment s's neighbours are s-1 and s+1 mod S, no point is held but the
    tile's two outermost ones, boundary b joins segments b and b+1 mod S and
    the trace is [ceil(K/T)][S][2]."""

    def __init__(self, u0, r, c1, cN, offsets, q, T, K, trace=None, stall=-1, limit_s=2.0, jitter_s=2e-4, seed=0,
                 periodic=False):
        self.u = np.array(u0, dtype=np.float64)
        self.periodic = bool(periodic)
        if not self.periodic:
            self.u[0], self.u[-1] = c1, cN
        self.N, self.r, self.q, self.T, self.K = len(self.u), float(r), int(q), int(T), int(K)
        self.off = [int(x) for x in offsets]
        self.S = len(self.off) - 1
        if self.off[0] != 0 or self.off[-1] != self.N:
            raise ValueError("offsets must run from 0 to N")
        inner = range(self.S) if self.periodic else range(1, self.S - 1)
        for s in inner:
            if self.off[s + 1] - self.off[s] < self.T:
                raise ValueError("segments with a neighbour on both sides need at least T points")
        if self.periodic and self.S < 2:
            raise ValueError("a ring needs at least two segments")
        self.R = 1
        while self.R < 2 * self.q:
            self.R *= 2
        self.nb = (self.K + self.T - 1) // self.T
        self.nbnd = self.S if self.periodic else self.S - 1  # boundaries
        self.trace_in = None if trace is None else np.asarray(trace, dtype=np.uint8).reshape(self.nb, self.nbnd, 2)
        self.trace = np.zeros((self.nb, max(self.nbnd, 0), 2), dtype=np.uint8)
        self.stall = stall
        self.limit_s = limit_s
        self.jitter_s = jitter_s
        self.seed = seed
        # strips[s][side][slot] = (version, points); side 0: first T points, 1: last T points
        self.strips = [[[(-1, None)] * self.R for _ in range(2)] for _ in range(self.S)]
        self.prog = [0] * self.S
        self.lock = threading.Lock()
        self.status = "ok"
        for s in range(self.S):
            lo, hi = self.off[s], self.off[s + 1]
            self.strips[s][0][0] = (0, self.u[lo:min(lo + self.T, hi)].copy())
            self.strips[s][1][0] = (0, self.u[max(hi - self.T, lo):hi].copy())
        self.max_lead = 0

    def _fail(self, what):
        with self.lock:
            if self.status == "ok":
                self.status = what

    def _read(self, nb, side, b, tidx, d_replay):
        need = b - min(d_replay, b) if d_replay is not None else max(b - self.q + 1, 0)
        if d_replay is not None and d_replay >= self.q:
            self._fail("trace")
            return None
        t0 = time.monotonic()
        while True:
            with self.lock:
                V = self.prog[nb]
                if self.status != "ok":
                    return None
                if V >= need:
                    v = need if d_replay is not None else min(V, b)
                    ver, pts = self.strips[nb][side][v % self.R]
                    if ver != v:
                        raise ProtocolError("segment read strip version %d from a slot holding version %d" % (v, ver))
                    if v > b:
                        raise ProtocolError("read a strip newer than the block")
                    self.trace[b][tidx[0]][tidx[1]] = b - v
                    return pts.copy()
            if time.monotonic() - t0 > self.limit_s:
                self._fail("timeout")
                return None
            time.sleep(0)

    def _neighbours(self, s):
        if self.periodic:
            return (s - 1) % self.S, (s + 1) % self.S
        return (s - 1 if s > 0 else -1), (s + 1 if s + 1 < self.S else -1)

    def _segment(self, s):
        rng = random.Random(self.seed * 1000 + s)
        lo, hi = self.off[s], self.off[s + 1]
        if self.periodic:  # the tile [lo - T, hi + T), indices mod N
            tlo, thi = lo - self.T, hi + self.T
        else:  # the tile [tlo, thi), clipped at the rod's ends
            tlo, thi = max(lo - self.T, 0), min(hi + self.T, self.N)
        sl, sr = self._neighbours(s)
        own = self.u[lo:hi].copy()
        for b in range(self.nb):
            if self.status != "ok":
                return
            if self.jitter_s:
                time.sleep(rng.random() * self.jitter_s)
            x = np.empty(thi - tlo)
            x[lo - tlo:hi - tlo] = own
            if sl >= 0:
                bnd = sl if self.periodic else s - 1  # boundary sl joins sl and s
                d = None if self.trace_in is None else int(self.trace_in[b][bnd][1])
                pts = self._read(sl, 1, b, (bnd, 1), d)
                if pts is None:
                    return
                x[:lo - tlo] = pts[len(pts) - (lo - tlo):]
            if sr >= 0:
                d = None if self.trace_in is None else int(self.trace_in[b][s][0])
                pts = self._read(sr, 0, b, (s, 0), d)
                if pts is None:
                    return
                x[hi - tlo:] = pts[:thi - hi]
            for _ in range(min(self.T, self.K - b * self.T)):
                y = x.copy()  # the tile's two outermost points are held
                y[1:-1] = self.r * ((x[2:] - 2.0 * x[1:-1]) + x[:-2]) + x[1:-1]
                if not self.periodic and tlo == 0:
                    y[0] = self.u[0]  # the Dirichlet ends (held)
                if not self.periodic and thi == self.N:
                    y[-1] = self.u[-1]
                x = y
            own = x[lo - tlo:hi - tlo].copy()
            if s == self.stall:
                continue  # never publishes
            with self.lock:
                slot = (b + 1) % self.R
                self.strips[s][0][slot] = (b + 1, own[:min(self.T, hi - lo)].copy())
                self.strips[s][1][slot] = (b + 1, own[max(hi - lo - self.T, 0):].copy())
                self.prog[s] = b + 1
                lead = max(((b + 1) - self.prog[n] for n in (sl, sr) if n >= 0), default=0)
                self.max_lead = max(self.max_lead, lead)
        with self.lock:
            self.u[lo:hi] = own

    def _segment_checked(self, s):
        try:
            self._segment(s)
        except ProtocolError as e:
            self._fail("protocol: %s" % e)

    def run(self):
        threads = [threading.Thread(target=self._segment_checked, args=(s,), daemon=True) for s in range(self.S)]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=self.limit_s * (self.nb + 10))
        return self.status
