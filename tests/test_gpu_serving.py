"""The continuous-batching server (amgdd_server_*): results alone and in a
mix of concurrent requests, batching, admission by device bytes with LRU
eviction, and the operator cache."""
import numpy as np
import pytest

from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK, seeded_rhs

from tests.test_gpu_parity import _rel

pytestmark = pytest.mark.gpu

OPS = [dict(N=24, theta=0.3, eps=1e-2), dict(N=32, theta=1.1, eps=1e-3), dict(N=40, theta=2.0, eps=1e-1)]
KW = dict(c_min=(2, 3), n_coarse=60)


@pytest.fixture(scope="module")
def amg():
    from paper_2601_04112_gb300 import build

    build.build()
    import paper_2601_04112_gb300 as amg

    amg.load_library()
    return amg


def _probs():
    return [q1_2d(o["N"], rotated_sqrtK(o["theta"], o["eps"]), agg=block_aggregates_2d(o["N"], 4)) for o in OPS]


def _requests(probs, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        k = int(rng.integers(len(probs)))
        nrhs = int(rng.integers(1, 4))
        out.append((k, seeded_rhs(probs[k].n, nrhs, 1000 * seed + j)))
    return out


def test_results_same_alone_and_in_the_mix(amg):
    probs = _probs()
    srv = amg.Server(slots=3)
    ops = [srv.add_operator(p, key=i, **KW)[0] for i, p in enumerate(probs)]
    reqs = _requests(probs, 30, 7)
    alone = []
    for k, B in reqs:  # one request in the system at a time
        x, infos, lat, st = srv.poll(srv.submit(ops[k], B))
        assert st == 0 and all(i["relres_true"] <= 1e-8 for i in infos)
        alone.append(x)
    s0 = srv.stats()
    rids = [srv.submit(ops[k], B) for k, B in reqs]  # all at once: they mix and batch
    for (k, B), rid, xa in zip(reqs, rids, alone):
        x, infos, lat, st = srv.poll(rid)
        assert st == 0 and all(i["status"] == 0 and i["relres_true"] <= 1e-8 for i in infos)
        # batched vs single solves differ only in summation order
        assert _rel(x, xa) <= 1e-9
        assert lat > 0.0
    s1 = srv.stats()
    cols_alone = sum(B.shape[1] for _, B in reqs)
    assert s1["completed"] == s0["completed"] + len(reqs)
    mix_batches = s1["batches"] - s0["batches"]
    # the mixed phase merged requests: fewer batches than requests
    assert mix_batches < len(reqs)
    assert cols_alone / mix_batches > cols_alone / len(reqs)
    assert s1["p99_ms"] >= s1["p50_ms"] > 0.0
    srv.close()


def test_budget_eviction_and_operator_cache(amg):
    probs = _probs()
    kw = dict(KW, tune=0)  # fixed kernel choices: footprints do not depend on timings
    sizes = []
    for p in probs:
        H = amg.Hierarchy.from_problem(p, overlap=1, **kw)
        sizes.append(H.device_bytes(with_batched=True))
        del H
    budget = sizes[1] + sizes[2] + sizes[0] // 2  # operators 1 and 2 fit together, not all three
    srv = amg.Server(hbm_budget=budget, slots=2)
    op0, c0 = srv.add_operator(probs[0], key=10, **kw)
    op1, c1 = srv.add_operator(probs[1], key=11, **kw)
    assert not c0 and not c1
    x, infos, _, st = srv.poll(srv.submit(op1, seeded_rhs(probs[1].n, 1, 3)))  # op1 now most recently used
    assert st == 0
    op2, c2 = srv.add_operator(probs[2], key=12, **kw)  # evicts op0, the least recently used idle one
    s = srv.stats()
    assert s["evictions"] == 1 and s["operators"] == 2 and s["device_bytes"] <= budget
    again, cached = srv.add_operator(probs[1], key=11, **kw)
    assert cached and again == op1
    with pytest.raises(amg.AmgddError):
        srv.submit(op0, seeded_rhs(probs[0].n, 1, 4))
    x, infos, _, st = srv.poll(srv.submit(op2, seeded_rhs(probs[2].n, 2, 5)))
    assert st == 0 and all(i["relres_true"] <= 1e-8 for i in infos)
    srv.close()


def test_mixed_precision_operators(amg):
    probs = _probs()
    srv = amg.Server(slots=2)
    ops = [srv.add_operator(p, key=20 + i, precision=amg.MIXED32, **KW)[0] for i, p in enumerate(probs)]
    rids = [srv.submit(ops[k], B) for k, B in _requests(probs, 12, 9)]
    for rid in rids:
        x, infos, lat, st = srv.poll(rid)
        assert st == 0 and all(i["relres_true"] <= 1e-8 for i in infos)
    srv.close()


def test_operators_built_on_the_request_path(amg):
    """Requests that carry their operator: one setup per distinct key, run by a worker; every result equals a
    solve of the same right-hand sides on a hierarchy built alone, to the batched solver's rounding."""
    probs = _probs()
    kw = dict(KW, tune=0)
    reqs = _requests(probs, 18, 11)
    refs = {}
    for k, p in enumerate(probs):
        H = amg.Hierarchy.from_problem(p, overlap=1, **kw)
        refs[k] = H
    expect = [np.asarray(refs[k].solve(B, tol=1e-8)[0]) for k, B in reqs]
    srv = amg.Server(slots=3)
    sub = [srv.submit_problem(probs[k], key=100 + k, b=B, **kw) for k, B in reqs]
    assert sum(not cached for _, cached in sub) == len({k for k, _ in reqs})
    for (rid, _), (k, B), xe in zip(sub, reqs, expect):
        x, infos, lat, st = srv.poll(rid)
        assert st == 0 and all(i["status"] == 0 and i["relres_true"] <= 1e-8 for i in infos)
        assert _rel(np.asarray(x).reshape(xe.shape), xe) <= 1e-9
    s = srv.stats()
    assert s["builds"] == len({k for k, _ in reqs}) and s["build_ms_total"] > 0.0
    assert s["bytes_per_unknown"] > 0.0
    srv.close()


def test_request_path_admission_waits_and_refuses(amg):
    """A budget that holds one operator at a time: requests of three operators built on the request path all
    complete, the idle operators being evicted between them; an operator larger than the whole budget fails
    its request with AMGDD_ERR_OOM instead of waiting forever."""
    probs = _probs()
    kw = dict(KW, tune=0)
    sizes = []
    for p in probs:
        H = amg.Hierarchy.from_problem(p, overlap=1, **kw)
        sizes.append(H.device_bytes(with_batched=True))
        del H
    srv = amg.Server(hbm_budget=int(max(sizes) * 1.6), slots=2)
    reqs = _requests(probs, 12, 13)
    sub = [srv.submit_problem(probs[k], key=200 + k, b=B, **kw) for k, B in reqs]
    for rid, _ in sub:
        x, infos, lat, st = srv.poll(rid)
        assert st == 0 and all(i["relres_true"] <= 1e-8 for i in infos)
    s = srv.stats()
    assert s["evictions"] >= 1 and s["device_bytes"] <= s["budget_bytes"]
    srv.close()
    tiny = amg.Server(hbm_budget=1 << 20, slots=1)
    rid, _ = tiny.submit_problem(probs[0], key=300, b=seeded_rhs(probs[0].n, 1, 1), **kw)
    with pytest.raises(amg.AmgddError) as e:
        tiny.poll(rid)
    assert e.value.status == -6
    tiny.close()
