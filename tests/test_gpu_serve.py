"""Serving: continuous batching of Dirac solves and force evaluations over
resident gauge fields of different volumes.  Results are checked against the
oracle, and each result is the same alone and inside a mix of requests."""
import numpy as np
import pytest
import torch

from tests import helpers as H

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module")
def serve():
    from paper_2602_20516_b300 import serve as S
    return S


def _full_canonical(field, dims):
    """(2, 12, Vh, 2) device field -> canonical (V, 4, 3) numpy."""
    from paper_2602_20516_b300 import lgt
    lat = lgt.Lattice(dims)
    return lat.unpack_spinor(field, lgt.FULL, lgt.FP64).cpu().numpy()


def _mom_canonical(field, dims):
    from paper_2602_20516_b300 import lgt
    lat = lgt.Lattice(dims)
    return lat.unpack_momenta(field).cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_and_force_vs_oracle(serve, ora, precision):
    srv = serve.Server(4 * GB, max_active=8, batch_iters=4)
    dims = (6, 4, 4, 8)
    g = srv.add_gauge(dims, 11, 0.5)
    Uo = ora.random_links(dims, 11, 0.5)          # the oracle draws the same field itself
    tol = 1e-12 if precision == "fp64" else 1e-10
    rs = srv.submit(g, serve.SOLVE, 0.15, precision, tol=tol, source_seed=5, keep_result=True)
    rf = srv.submit(g, serve.FORCE, 0.15, precision, tol=tol, source_seed=6, beta=5.8, keep_result=True)
    done = {c["id"]: c for c in srv.run_until_idle()}
    assert done[rs]["status"] == 0 and done[rf]["status"] == 0
    bar = 1e-9 if precision == "fp64" else 1e-6
    # solve: x = D^{-1} b, b from Philox (source field)
    b = ora.gaussian_spinor(dims, 5, 0, ora.FIELD_SOURCE, 3)
    xo, _, _ = ora.cg(dims, Uo, 0.15, ora.dirac(dims, Uo, 0.15, b, dagger=True), tol=1e-13)
    x = _full_canonical(srv.result(rs), dims)
    assert H.rel(x, xo) < bar
    # force: gauge + even-odd pseudofermion force with phi_e from Philox
    phi = ora.gaussian_spinor(dims, 6, 0, ora.FIELD_SOURCE, 1)
    Fo = ora.gauge_force(dims, Uo, 5.8) + ora.pf_force(dims, Uo, 0.15, phi, eo=True, tol=1e-13)[0]
    F = _mom_canonical(srv.result(rf), dims)
    assert H.rel(F, Fo) < bar
    srv.close()


def test_mixed_requests_with_and_without_double_float_copy(serve, ora):
    """A mixed request forms its true residuals (and a force request its forces) in
    double-float when its gauge field has a double-float copy, which the server makes
    while the gauge fields with copies stay within half the budget; otherwise it uses
    the FP64 hop and FP64 forces.  Both meet the tolerance, agree with the oracle
    within the solve's error bound (cond(A) ~ 1e2 times tol 1e-10) and with each
    other."""
    dims = (6, 4, 4, 8)
    Vh = int(np.prod(dims)) // 2
    links64, links12 = 8 * 9 * Vh * 16, 8 * 3 * Vh * 16
    res = {}
    for name, budget in (("df", 4 * GB), ("fp64", 2_000_000)):
        srv = serve.Server(budget, max_active=4, batch_iters=4)
        g = srv.add_gauge(dims, 11, 0.5)
        assert srv.info()["used_bytes"] == links64 + links12 + (links64 if name == "df" else 0)
        out = []
        # one at a time: a kept result holds its memory until fetched, and under the
        # small budget only one request fits
        for kind, seed, conv in ((serve.SOLVE, 5, _full_canonical), (serve.FORCE, 6, _mom_canonical)):
            r = srv.submit(g, kind, 0.15, "mixed", tol=1e-10, source_seed=seed, beta=5.8, keep_result=True)
            done = {c["id"]: c for c in srv.run_until_idle()}
            assert done[r]["status"] == 0 and done[r]["true_rel_residual"] <= 1e-10, (name, done[r])
            out.append(conv(srv.result(r), dims))
        res[name] = tuple(out)
        srv.close()
    Uo = ora.random_links(dims, 11, 0.5)
    b = ora.gaussian_spinor(dims, 5, 0, ora.FIELD_SOURCE, 3)
    xo, _, _ = ora.cg(dims, Uo, 0.15, ora.dirac(dims, Uo, 0.15, b, dagger=True), tol=1e-13)
    phi = ora.gaussian_spinor(dims, 6, 0, ora.FIELD_SOURCE, 1)
    Fo = ora.gauge_force(dims, Uo, 5.8) + ora.pf_force(dims, Uo, 0.15, phi, eo=True, tol=1e-13)[0]
    for name, (x, F) in res.items():
        assert H.rel(x, xo) < 1e-7 and H.rel(F, Fo) < 1e-7, name
    assert H.rel(res["df"][0], res["fp64"][0]) < 1e-7 and H.rel(res["df"][1], res["fp64"][1]) < 1e-7


def test_result_same_alone_and_in_mix(serve):
    """A request's result is bitwise identical whether it runs alone or batched
    with requests of other volumes and precisions arriving around it."""
    dims_list = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32), (8, 8, 8, 16)]
    probes = [dict(kind=serve.SOLVE, kappa=0.152, precision="mixed", tol=1e-10, source_seed=101),
              dict(kind=serve.FORCE, kappa=0.149, precision="fp64", tol=1e-10, source_seed=102, beta=5.8)]
    alone = []
    for p in probes:
        srv = serve.Server(16 * GB, max_active=32, batch_iters=8)
        gids = [srv.add_gauge(d, 20 + k, 0.45) for k, d in enumerate(dims_list)]
        rid = srv.submit(gids[1], keep_result=True, **p)
        srv.run_until_idle()
        alone.append(srv.result(rid).clone())
        srv.close()
    srv = serve.Server(16 * GB, max_active=32, batch_iters=8)
    gids = [srv.add_gauge(d, 20 + k, 0.45) for k, d in enumerate(dims_list)]
    mix = serve.workload(gids, 24, seed=3)
    ids = []
    for k, r in enumerate(mix):
        srv.submit(**r)
        if k == 5:
            ids.append(srv.submit(gids[1], keep_result=True, **probes[0]))
        if k % 6 == 0:
            srv.step()
        if k == 17:
            ids.append(srv.submit(gids[1], keep_result=True, **probes[1]))
    done = srv.run_until_idle()
    assert all(c["status"] == 0 for c in done)
    for rid, ref in zip(ids, alone):
        assert torch.equal(srv.result(rid), ref)
    srv.close()


def test_budget_admission_and_refusal(serve):
    """Under a tight budget requests wait for memory and all finish; a request that
    can never fit is refused with LGT_ENOMEM."""
    srv = serve.Server(int(0.25 * GB), max_active=16, batch_iters=8)
    g_small = srv.add_gauge((8, 8, 8, 8), 1, 0.4)
    g_mid = srv.add_gauge((16, 16, 16, 16), 2, 0.4)
    for k in range(12):
        srv.submit(g_mid if k % 2 else g_small, serve.SOLVE, 0.15, "mixed", source_seed=k + 1)
    peak_active, peak_used = 0, 0
    done = []
    while True:
        a, q = srv.step()
        info = srv.info()
        peak_active = max(peak_active, a)
        peak_used = max(peak_used, info["used_bytes"])
        done += srv.poll()
        if a == 0 and q == 0:
            break
    assert len(done) == 12 and all(c["status"] == 0 for c in done)
    assert peak_used <= 0.25 * GB and peak_active < 12
    srv.close()
    # 4 MiB: the 8^4 gauge field (3.1 MiB) fits, a force request (~6 MiB) never can
    tiny = serve.Server(4 << 20, max_active=4, batch_iters=4)
    g = tiny.add_gauge((8, 8, 8, 8), 1, 0.4)
    tiny.submit(g, serve.FORCE, 0.15, "fp64", source_seed=1, beta=5.8)
    done = tiny.run_until_idle()
    assert len(done) == 1 and done[0]["status"] == 2   # LGT_ENOMEM
    tiny.close()


def test_poisson_latency_smoke(serve):
    srv = serve.Server(8 * GB, max_active=32, batch_iters=8)
    gids = [srv.add_gauge(d, 30 + k, 0.5) for k, d in enumerate([(8, 8, 8, 8), (12, 12, 12, 12)])]
    reqs = serve.workload(gids, 40, seed=9)
    thr, _ = serve.saturated(srv, reqs)
    done = serve.poisson(srv, serve.workload(gids, 60, seed=10), 0.5 * thr, seed=11, warmup=5)
    st = serve.latency_stats(done)
    assert st["n"] == 55 and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_near_critical_mixed_requests_succeed(serve):
    """Smooth fields (alpha 0.3) with kappa at the top of the request range make
    Dhat^+ Dhat nearly singular; FP32 rounding can then break the mixed CG recursion
    (<p, A p> <= 0) or stall it.  The server restarts such a request from its FP64
    residual (and hands a stalled one over to FP64 CG), so every request completes, to
    its tolerance, with the solution of the FP64 request."""
    srv = serve.Server(8 * GB, max_active=16, batch_iters=4)
    dims = (8, 8, 8, 8)
    g = [srv.add_gauge(dims, 20 + k, 0.3) for k in range(2)]
    reqs = {}
    for k, kappa in enumerate((0.150, 0.155, 0.157)):
        for gi in g:
            for prec in ("mixed", "fp64"):
                rid = srv.submit(gi, serve.SOLVE, kappa, prec, tol=1e-10, source_seed=40 + k, keep_result=True)
                reqs[rid] = (gi, kappa, prec)
    done = {c["id"]: c for c in srv.run_until_idle()}
    for rid, (gi, kappa, prec) in reqs.items():
        assert done[rid]["status"] == 0, (gi, kappa, prec, done[rid])
        assert done[rid]["true_rel_residual"] <= 1e-10
    for rid, (gi, kappa, prec) in reqs.items():
        if prec != "mixed":
            continue
        twin = next(r for r, v in reqs.items() if v == (gi, kappa, "fp64"))
        a, b = srv.result(rid), srv.result(twin)
        assert (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item() < 1e-6, (gi, kappa)
    srv.close()
