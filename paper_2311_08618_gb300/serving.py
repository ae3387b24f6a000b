"""Continuous-batching server for k-th eigenvalue queries against resident,
factor-ready H^2 matrices (a scheduling layer above the C ABI; every inertia
evaluation runs in the library's CUDA kernels).

Model
-----
* Each resident matrix owns a handle whose workspace holds ``lanes`` shifted
  factorizations at once (its HBM footprint, ``h2_info()['workspace_bytes']``).
  A request occupies at least one lane per round; a matrix admits new
  requests only while it has a free lane, so what is in flight never
  exceeds the memory reserved for it (admission by HBM footprint).
* A tick runs one multisection round on every matrix with active requests:
  the distinct active intervals of that matrix share its lanes (q interior
  points each).  When the resident matrices share max_lanes and precision,
  the round of all of them is one group batch (h2_group: one launch per tree
  level and colour over all matrices, idle ones with no shifts); otherwise
  their batches are enqueued back to back on the server's CUDA stream.  The
  tick waits once, then every interval of every request is narrowed with
  all (mu, nu) pairs of its matrix's round (Algorithm 1; inertia reuse across
  requests, Sec. 4.2).  Requests of one matrix share its batch, so their work
  overlaps on the device.  (Giving every matrix its own stream stalled the
  device in testing: all started kernels completed, yet a queued one never
  started; one stream avoids it.)
* Requests that arrive while others are on the GPU join at the next tick
  (continuous batching).  A new request starts from the tightest bracket in
  its matrix's table of evaluated (mu, nu) pairs instead of the Gershgorin
  interval (Sec. 4.2).
* A request completes when its bracket is narrower than its tol; the result
  is the midpoint, with |lambda_k - result| < tol/2 (Eq. error-bound).
"""
from __future__ import annotations

import bisect
import ctypes as C
import time
from dataclasses import dataclass, field

import numpy as np

from .binding import H2Group, H2Matrix, lib


@dataclass
class Request:
    rid: int
    matrix: str
    k: int
    tol: float
    t_arrival: float
    lo: float = 0.0
    hi: float = 0.0
    t_done: float = -1.0
    result: float = float("nan")
    rounds: int = 0


@dataclass
class _Resident:
    name: str
    h2: H2Matrix
    lanes: int
    stream: object
    lo0: float
    hi0: float
    precision: int = 0
    table_mu: list = field(default_factory=list)      # sorted evaluated shifts
    table_nu: list = field(default_factory=list)
    active: list = field(default_factory=list)
    d_shifts: object = None
    d_counts: object = None
    h_shifts: object = None
    h_counts: object = None


def plan_shifts(intervals, lanes):
    """The shifts of one round on one matrix: the first `lanes` distinct
    intervals (in order) share its lanes, each cut at q equally spaced
    interior points ((q+1)-section, Algorithm 1 with spare lanes)."""
    ivs = []
    seen = set()
    for key in intervals:
        if key not in seen:
            seen.add(key)
            ivs.append(key)
    if not ivs:
        return []
    m = min(len(ivs), lanes)
    q, extra = divmod(lanes, m)
    shifts = []
    for u in range(m):
        a, b = ivs[u]
        qu = q + (1 if u < extra else 0)
        shifts += [a + (b - a) * j / (qu + 1) for j in range(1, qu + 1)]
    return shifts


def narrow(lo, hi, k, shifts, counts):
    """[lo, hi] narrowed by every evaluated (mu, nu) inside it: nu >= k moves
    hi down to mu, nu < k moves lo up to mu (Algorithm 1)."""
    for mu, nu in zip(shifts, counts):
        if lo < mu < hi:
            if nu >= k:
                hi = mu
            else:
                lo = mu
    return lo, hi


def tightest_bracket(lo0, hi0, table_mu, table_nu, k):
    """The tightest [mu_lo, mu_hi] with nu(mu_lo) < k <= nu(mu_hi) in a table
    of evaluated (mu, nu) pairs, starting from [lo0, hi0] (Sec. 4.2)."""
    lo, hi = lo0, hi0
    for mu, nu in zip(table_mu, table_nu):
        if nu < k:
            lo = max(lo, mu)
        else:
            hi = min(hi, mu)
    return lo, hi


class Server:
    """Resident matrices + request queue + continuous batching (see module doc)."""

    def __init__(self, hbm_budget_bytes: int | None = None):
        import torch
        self.torch = torch
        self.mats: dict[str, _Resident] = {}
        self.queue: list[Request] = []
        self.done: list[Request] = []
        self.next_id = 0
        self.budget = hbm_budget_bytes
        self.footprint = 0
        self.shifts_evaluated = 0
        self.ticks = 0
        self.stream = torch.cuda.Stream()       # one stream for all resident matrices
        self.group = None                       # group batch over all resident matrices
        self._group_dirty = True
        self.host_s = 0.0                       # time spent planning and narrowing on the host
        self.wait_s = 0.0                       # time spent waiting for the device's batches

    # -- residency ----------------------------------------------------------
    def add_matrix(self, name, points, kernel, kparams, leaf, rank, eta=1.0, lanes=16, **opts):
        """Builds and keeps resident an H^2 matrix; refuses it when the HBM
        budget would be exceeded by its workspace."""
        torch = self.torch
        stream = self.stream
        h = H2Matrix(points, kernel, kparams, leaf=leaf, rank=rank, eta=eta, max_lanes=lanes,
                     stream=stream.cuda_stream, **opts)
        info = h.h2_info()
        if self.budget is not None and self.footprint + info["workspace_bytes"] > self.budget:
            h.close()
            raise MemoryError("matrix %s does not fit the HBM budget" % name)
        self.footprint += info["workspace_bytes"]
        a = info["gershgorin_lo"] - 1e-6 * info["norm_inf"]
        b = info["gershgorin_hi"] + 1e-6 * info["norm_inf"]
        r = _Resident(name, h, lanes, stream, a, b, int(opts.get("precision", 0)))
        r.d_shifts = torch.zeros(lanes, dtype=torch.float64, device="cuda")
        r.d_counts = torch.zeros(lanes, dtype=torch.int64, device="cuda")
        r.h_shifts = torch.zeros(lanes, dtype=torch.float64).pin_memory()
        r.h_counts = torch.zeros(lanes, dtype=torch.int64).pin_memory()
        # the table starts with the interval ends: nu(a) = 0, nu(b) = n
        r.table_mu = [a, b]
        r.table_nu = [0, h.n]
        self.mats[name] = r
        self._group_dirty = True
        return info

    def _ensure_group(self):
        """The group of all resident matrices (None if their lanes or
        precisions differ), with its shift and count buffers."""
        if not self._group_dirty:
            return self.group
        torch = self.torch
        if self.group is not None:
            self.group.close()
            self.group = None
        mats = list(self.mats.values())
        lanes = {r.h2.h2_info()["lanes"] for r in mats}
        opts_ok = len(lanes) == 1 and len({r.precision for r in mats}) == 1
        if mats and opts_ok:
            self.group = H2Group([r.h2 for r in mats])
            L = mats[0].lanes
            self.g_order = [r.name for r in mats]
            self.g_hsh = torch.zeros((len(mats), L), dtype=torch.float64).pin_memory()
            self.g_hc = torch.zeros((len(mats), L), dtype=torch.int64).pin_memory()
            self.g_dsh = torch.zeros((len(mats), L), dtype=torch.float64, device="cuda")
            self.g_dc = torch.zeros((len(mats), L), dtype=torch.int64, device="cuda")
        self._group_dirty = False
        return self.group

    def close(self):
        if self.group is not None:
            self.group.close()
            self.group = None
        for r in self.mats.values():
            r.h2.close()
        self.mats.clear()

    # -- requests -------------------------------------------------------------
    def submit(self, matrix: str, k: int, tol: float, t_arrival: float | None = None) -> int:
        if matrix not in self.mats:
            raise KeyError(matrix)
        r = self.mats[matrix]
        if not 1 <= k <= r.h2.n:
            raise ValueError("k out of range")
        req = Request(self.next_id, matrix, int(k), float(tol),
                      time.perf_counter() if t_arrival is None else t_arrival)
        self.next_id += 1
        self.queue.append(req)
        return req.rid

    def poll(self) -> list[Request]:
        out, self.done = self.done, []
        return out

    def busy(self) -> bool:
        return bool(self.queue) or any(r.active for r in self.mats.values())

    def _bracket(self, r: _Resident, k: int):
        """Tightest [mu_lo, mu_hi] from the (mu, nu) table: nu(mu_lo) < k <= nu(mu_hi)."""
        return tightest_bracket(r.lo0, r.hi0, r.table_mu, r.table_nu, k)

    def _admit(self):
        keep = []
        for req in self.queue:
            r = self.mats[req.matrix]
            if len(r.active) < r.lanes:          # a free lane slot
                req.lo, req.hi = self._bracket(r, req.k)
                if req.hi - req.lo < req.tol:
                    self._finish(req)
                else:
                    r.active.append(req)
            else:
                keep.append(req)
        self.queue = keep

    def _finish(self, req: Request):
        req.result = 0.5 * (req.lo + req.hi)
        req.t_done = time.perf_counter()
        self.done.append(req)

    # -- one tick ---------------------------------------------------------------
    def step(self):
        """Admit, run one multisection round on every busy matrix, update."""
        t_host = time.perf_counter()
        self._admit()
        plans = {}
        for r in self.mats.values():
            if not r.active:
                continue
            # distinct active intervals share the lanes
            plans[r.name] = plan_shifts([(req.lo, req.hi) for req in r.active], r.lanes)
        if not plans:
            self.ticks += 1
            return 0
        G = self._ensure_group()
        results = {}
        if G is not None:
            ns = []
            for i, name in enumerate(self.g_order):
                sh = plans.get(name, [])
                ns.append(len(sh))
                if sh:
                    self.g_hsh[i, :len(sh)] = self.torch.tensor(sh, dtype=self.torch.float64)
            with self.torch.cuda.stream(self.stream):
                self.g_dsh.copy_(self.g_hsh, non_blocking=True)
                G.h2_group_inertia_device(self.g_dsh, ns, self.g_dc)
                self.g_hc.copy_(self.g_dc, non_blocking=True)
            t_w = time.perf_counter()
            self.stream.synchronize()
            self.wait_s += time.perf_counter() - t_w
            hc = self.g_hc.numpy()
            for i, name in enumerate(self.g_order):
                if ns[i]:
                    results[name] = hc[i, :ns[i]].copy()
        else:
            L = lib()
            for name, shifts in plans.items():
                r = self.mats[name]
                ns = len(shifts)
                r.h_shifts[:ns] = self.torch.tensor(shifts, dtype=self.torch.float64)
                with self.torch.cuda.stream(r.stream):
                    r.d_shifts[:ns].copy_(r.h_shifts[:ns], non_blocking=True)
                    rc = L.h2_inertia_device(r.h2._h, C.c_void_p(r.d_shifts.data_ptr()), ns,
                                             C.c_void_p(r.d_counts.data_ptr()), None)
                    if rc != 0:
                        raise RuntimeError(L.h2_last_error().decode())
                    r.h_counts[:ns].copy_(r.d_counts[:ns], non_blocking=True)
            t_w = time.perf_counter()
            self.stream.synchronize()
            self.wait_s += time.perf_counter() - t_w
            for name, shifts in plans.items():
                results[name] = self.mats[name].h_counts[:len(shifts)].numpy().copy()
        for name, shifts in plans.items():
            r = self.mats[name]
            counts = results[name]
            self.shifts_evaluated += len(shifts)
            for mu, nu in zip(shifts, counts):
                i = bisect.bisect_left(r.table_mu, mu)
                r.table_mu.insert(i, mu)
                r.table_nu.insert(i, int(nu))
            still = []
            for req in r.active:
                req.lo, req.hi = narrow(req.lo, req.hi, req.k, shifts, counts)
                req.rounds += 1
                if req.hi - req.lo < req.tol:
                    self._finish(req)
                else:
                    still.append(req)
            r.active = still
        self.ticks += 1
        self.host_s += time.perf_counter() - t_host
        return len(plans)


def run_open_loop(server: Server, arrivals, horizon_s: float, deadline_s: float):
    """Replays (t_offset, matrix, k, tol) arrivals in wall-clock time while
    ticking the server until all are done or deadline_s has passed (then the
    queue and the active requests are dropped and counted as unfinished).
    Returns (completed requests, number unfinished)."""
    t0 = time.perf_counter()
    arrivals = sorted(arrivals)
    i = 0
    done = []
    while True:
        now = time.perf_counter() - t0
        if now > deadline_s:
            unfinished = len(server.queue) + sum(len(r.active) for r in server.mats.values()) + \
                (len(arrivals) - i)
            server.queue = []
            for r in server.mats.values():
                r.active = []
            return done + server.poll(), unfinished
        while i < len(arrivals) and arrivals[i][0] <= now:
            ta, m, k, tol = arrivals[i]
            server.submit(m, k, tol, t_arrival=t0 + ta)
            i += 1
        if server.busy():
            server.step()
        elif i < len(arrivals):
            time.sleep(max(0.0, min(1e-3, arrivals[i][0] - now)))
        else:
            break
        done += server.poll()
        if now > horizon_s and not server.busy() and i >= len(arrivals):
            break
    done += server.poll()
    return done, 0


def latency_stats(done):
    lat = np.array([r.t_done - r.t_arrival for r in done])
    if lat.size == 0:
        return {}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}
