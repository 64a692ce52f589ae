"""Serving front end: a request server over resident gauge fields (C ABI
lgt_server_*) and a Poisson load generator reporting latency percentiles.

The scheduling (admission by HBM budget, batched CG iterations across requests,
reliable updates, epilogues) runs in liblgt; this module marshals arguments and
drives the clock.
"""
import ctypes as C
import collections
import time

import numpy as np
import torch

from . import lgt

SOLVE, FORCE = lgt.REQ_SOLVE, lgt.REQ_FORCE


class Server:
    def __init__(self, hbm_budget_bytes, max_active=64, batch_iters=8, delta=1e-3, torch_allocator=True):
        if not torch.cuda.is_available():
            raise RuntimeError("the server needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream(self.device)
        self._keep = []
        alloc = None
        if torch_allocator:
            dev = self.device.index

            def _a(ctx, nbytes, st):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st or 0)
                except RuntimeError:
                    return None

            def _f(ctx, ptr, st):
                torch.cuda.caching_allocator_delete(ptr)

            alloc = lgt.Allocator(lgt.ALLOC_FN(_a), lgt.FREE_FN(_f), None)
            self._keep.append(alloc)
        h = C.c_void_p()
        lgt.check(lgt.lib().lgt_server_create(C.byref(alloc) if alloc else None, int(hbm_budget_bytes), max_active,
                                              batch_iters, delta, C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.dims = {}
        self.kinds = {}

    def close(self):
        if getattr(self, "h", None):
            lgt.lib().lgt_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_gauge(self, dims, seed, alpha):
        gid = C.c_int()
        lgt.check(lgt.lib().lgt_server_add_gauge(self.h, (C.c_int * 4)(*dims), seed, alpha, C.byref(gid)))
        self.dims[gid.value] = tuple(dims)
        return gid.value

    def links(self, gauge_id):
        V = int(np.prod(self.dims[gauge_id]))
        U = torch.zeros((V, 4, 3, 3), dtype=torch.complex128, device=self.device)
        lgt.check(lgt.lib().lgt_server_get_links(self.h, gauge_id, C.c_void_p(U.data_ptr())))
        return U

    def submit(self, gauge_id, kind, kappa, precision="fp64", tol=1e-10, source_seed=0, beta=0.0,
               max_iter=10000, keep_result=False):
        prec = {"fp64": lgt.FP64, "mixed": lgt.MIXED}[precision] if isinstance(precision, str) else precision
        q = lgt.Request(gauge_id, kind, prec, kappa, beta, tol, max_iter, source_seed, int(keep_result))
        rid = C.c_uint64()
        lgt.check(lgt.lib().lgt_server_submit(self.h, C.byref(q), C.byref(rid)))
        self.kinds[rid.value] = (gauge_id, kind)
        return rid.value

    def step(self):
        a, q = C.c_int(), C.c_int()
        lgt.check(lgt.lib().lgt_server_step(self.h, C.byref(a), C.byref(q)))
        return a.value, q.value

    def poll(self, max_n=4096):
        buf = (lgt.Completion * max_n)()
        n = C.c_int()
        lgt.check(lgt.lib().lgt_server_poll(self.h, buf, max_n, C.byref(n)))
        return [buf[k].as_dict() for k in range(n.value)]

    def result(self, rid):
        gid, kind = self.kinds[rid]
        Vh = int(np.prod(self.dims[gid])) // 2
        shape = (2, 12, Vh, 2) if kind == SOLVE else (2, 4, 4, Vh, 2)
        out = torch.zeros(shape, dtype=torch.float64, device=self.device)
        lgt.check(lgt.lib().lgt_server_result(self.h, rid, C.c_void_p(out.data_ptr()), out.numel() * 8))
        return out

    def info(self):
        u, b, a, q = C.c_size_t(), C.c_size_t(), C.c_int(), C.c_int()
        lgt.check(lgt.lib().lgt_server_info(self.h, C.byref(u), C.byref(b), C.byref(a), C.byref(q)))
        return {"used_bytes": u.value, "budget_bytes": b.value, "active": a.value, "queued": q.value}

    def run_until_idle(self, max_steps=1000000):
        done = []
        for _ in range(max_steps):
            a, q = self.step()
            done += self.poll()
            if a == 0 and q == 0:
                done += self.poll()
                return done
        raise RuntimeError("server did not drain")


def clock():
    return lgt.lib().lgt_clock()


def workload(gauges, n, seed, solve_fraction=0.7, kappa=(0.14, 0.157), mixed_fraction=0.5, tol=1e-10, beta=5.8):
    """Request mix: Dirac solves and force evaluations on randomly chosen resident
    gauge fields, kappa uniform in the range, FP64 / mixed split."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        out.append(dict(gauge_id=int(rng.choice(gauges)),
                        kind=SOLVE if rng.random() < solve_fraction else FORCE,
                        kappa=float(rng.uniform(*kappa)),
                        precision="mixed" if rng.random() < mixed_fraction else "fp64",
                        tol=tol, source_seed=int(rng.integers(1, 2 ** 62)), beta=beta))
    return out


def saturated(server, reqs):
    """Submit everything at once and drain: requests per second."""
    t0 = clock()
    for r in reqs:
        server.submit(**r)
    done = server.run_until_idle()
    return len(reqs) / (clock() - t0), done


def poisson(server, reqs, rate, seed, warmup=0):
    """Open-loop Poisson arrivals at `rate` requests/s; latency = completion time -
    scheduled arrival time (queueing included).  Returns the completions of the
    requests after the first `warmup`, with a 'latency' key."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, len(reqs))
    t0 = clock() + 0.01
    arrival = t0 + np.cumsum(gaps)
    ids = {}
    k = 0
    done = []
    while k < len(reqs) or server.info()["active"] or server.info()["queued"]:
        now = clock()
        while k < len(reqs) and arrival[k] <= now:
            ids[server.submit(**reqs[k])] = k
            k += 1
        a, q = server.step()
        done += server.poll()
        if a == 0 and q == 0 and k < len(reqs):
            # idle until the next arrival
            wait = arrival[k] - clock()
            if wait > 0:
                time.sleep(min(wait, 0.01))
    done += server.poll()
    out = []
    for c in done:
        i = ids[c["id"]]
        if i < warmup:
            continue
        c = dict(c)
        c["latency"] = c["t_done"] - arrival[i]
        c["queued"] = c["t_admit"] - arrival[i]
        c["index"] = i
        c["gauge_id"] = reqs[i]["gauge_id"]
        c["kind"] = reqs[i]["kind"]
        c["precision"] = reqs[i]["precision"]
        out.append(c)
    return out


def _pct(a, q):
    return 1e3 * float(np.percentile(a, q)) if len(a) else None


def latency_stats(done):
    """p50 / p99 / mean latency of the successful completions (failed requests are
    excluded from these and counted apart), and p99 over every completion."""
    ok = np.array([c["latency"] for c in done if c["status"] == 0])
    allc = np.array([c["latency"] for c in done])
    if ok.size == 0:
        return {"p50_ms": None, "p99_ms": None, "n": 0, "failed": len(done)}
    return {"p50_ms": _pct(ok, 50), "p99_ms": _pct(ok, 99),
            "mean_ms": 1e3 * float(ok.mean()), "n": int(ok.size),
            "p99_all_completions_ms": _pct(allc, 99), "failures_excluded_from_percentiles": True,
            "failed": int(sum(1 for c in done if c["status"] != 0)),
            "failed_by_status": {str(k): v for k, v in
                                 collections.Counter(c["status"] for c in done if c["status"] != 0).items()}}


def latency_breakdown(done, label):
    """Latency percentiles per class label(c) (e.g. volume, kind, precision), with the
    time spent queued (arrival -> admission) and served (admission -> completion)."""
    groups = collections.defaultdict(list)
    for c in done:
        if c["status"] == 0:
            groups[label(c)].append(c)
    out = {}
    for k, cs in sorted(groups.items()):
        lat = np.array([c["latency"] for c in cs])
        q = np.array([c.get("queued", 0.0) for c in cs])
        out[k] = {"n": len(cs), "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
                  "queued_p50_ms": _pct(q, 50), "served_p50_ms": _pct(lat - q, 50),
                  "served_p99_ms": _pct(lat - q, 99),
                  "iters_mean": float(np.mean([c["iters"] for c in cs]))}
    return out
