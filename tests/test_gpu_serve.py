"""Serving runtime on the GPU: continuous batching over resident clouds.

Each request's result must be the same alone and in the mix: every request
of a mixed, concurrently submitted workload (queries, gradients, Booleans,
trace steps, offsets; host and device buffers; three submitting threads; one
stream priority, or small requests on high-priority streams) is
compared bit for bit with the same request run alone on a one-slot server,
and (except trace steps) with the direct calls; a weighted cloud and
log-sum-exp queries likewise.  Admission is checked under a one-slot budget,
oversized requests are refused, and a poll can time out.
"""
import threading

import numpy as np
import pytest

import synth
from workloads import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_16946_b300 import build
    build.build()
    import paper_2607_16946_b300 as m
    from paper_2607_16946_b300 import serve
    clouds = [m.Cloud(*f32(*synth.sphere_fibonacci(3000, 1))),
              m.Cloud(*f32(*synth.ring_torus(20000, 2))),
              m.Cloud(*f32(*synth.ellipsoid(8000, 3))),
              m.Cloud(*f32(*synth.superquadric(12000, 4, grid=256)))]
    return m, serve, torch, clouds


def alone(m, torch, clouds, kind, ca, cb, x, dirs=None, t=None, offset=0.0):
    from paper_2607_16946_b300 import serve as S
    c = clouds[ca]
    if kind == S.SDF_REQ_QUERY:
        return c.query(x, offset=offset)
    if kind == S.SDF_REQ_GRAD:
        phi, g, _ = c.query_grad(x, saved=False, offset=offset)
        return torch.cat([phi, g.reshape(-1)])
    a = c.query(x, offset=offset)
    b = clouds[cb].query(x, offset=offset)
    op = {S.SDF_REQ_UNION: m.SDF_UNION, S.SDF_REQ_INTERSECT: m.SDF_INTERSECT,
          S.SDF_REQ_DIFFERENCE: m.SDF_DIFFERENCE}[kind]
    return m.combine(op, a, b)


@pytest.mark.parametrize("express", [0.0, 0.5])
def test_mixed_requests_equal_alone(env, express):
    """express = 0.5: requests of at most 5e8 pairs (about half of this mix)
    on two high-priority streams, the others on two low-priority ones."""
    m, S, torch, clouds = env
    srv = S.Server(mem_budget_bytes=2 << 30, max_inflight=6, n_streams=4, express_gpairs=express)
    ids = [srv.register(c) for c in clouds]
    rng = np.random.Generator(np.random.PCG64(11))
    reqs = []
    for i in range(48):
        kind = int(rng.choice([S.SDF_REQ_QUERY] * 4 + [S.SDF_REQ_GRAD, S.SDF_REQ_UNION, S.SDF_REQ_INTERSECT,
                                                        S.SDF_REQ_DIFFERENCE, S.SDF_REQ_TRACE_STEP]))
        q = int(np.exp(rng.uniform(np.log(100), np.log(60000))))
        x = torch.as_tensor(f32(rng.uniform(-1.5, 1.5, size=(q, 3))), dtype=torch.float32, device="cuda")
        dirs = t = None
        if kind == S.SDF_REQ_TRACE_STEP:
            d = synth._unit(rng.normal(size=(q, 3)))
            dirs = torch.as_tensor(f32(d), dtype=torch.float32, device="cuda")
            t = torch.as_tensor(f32(rng.uniform(0, 0.5, size=q)), dtype=torch.float32, device="cuda")
        host = bool(rng.integers(0, 2)) and kind != S.SDF_REQ_TRACE_STEP
        nout = 4 * q if kind == S.SDF_REQ_GRAD else q
        out = np.empty(nout, np.float32) if host else torch.empty(nout, device="cuda")
        xin = x.cpu().numpy() if host else x
        offset = float(rng.choice([0.0, 0.05]))
        reqs.append(dict(kind=kind, ca=int(rng.integers(0, 4)), cb=int(rng.integers(0, 4)), x=x, xin=xin,
                         dirs=dirs, t=t, out=out, offset=offset))
    torch.cuda.synchronize()
    tickets = [None] * len(reqs)

    def submitter(k):
        for i in range(k, len(reqs), 3):
            r = reqs[i]
            tickets[i] = srv.submit(r["kind"], ids[r["ca"]], r["xin"], r["out"], cloud_id_b=ids[r["cb"]],
                                    dirs=r["dirs"], t=r["t"], offset=r["offset"])

    th = [threading.Thread(target=submitter, args=(k,)) for k in range(3)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    stats = [srv.poll(tk) for tk in tickets]
    srv.shutdown()
    # the same requests one at a time through a one-slot server
    solo = S.Server(mem_budget_bytes=2 << 30, max_inflight=1, n_streams=1)
    sid = [solo.register(c) for c in clouds]
    for r, st in zip(reqs, stats):
        got = r["out"] if isinstance(r["out"], np.ndarray) else r["out"].cpu().numpy()
        out1 = np.empty_like(got) if isinstance(r["out"], np.ndarray) else torch.empty_like(r["out"])
        solo.poll(solo.submit(r["kind"], sid[r["ca"]], r["xin"], out1, cloud_id_b=sid[r["cb"]],
                              dirs=r["dirs"], t=r["t"], offset=r["offset"]))
        one = out1 if isinstance(out1, np.ndarray) else out1.cpu().numpy()
        np.testing.assert_array_equal(got, one)
        if r["kind"] != S.SDF_REQ_TRACE_STEP:      # and equal to the direct calls
            ref = alone(m, torch, clouds, r["kind"], r["ca"], r["cb"], r["x"], offset=r["offset"])
            np.testing.assert_array_equal(got, ref.cpu().numpy())
        assert st["arrive_ns"] <= st["admit_ns"] <= st["start_ns"] <= st["done_ns"]
    solo.shutdown()


def test_smallest_first_admission(env):
    """SMALLEST_FIRST: with one slot busy on a large request, queued requests
    are admitted smallest first; results are unchanged."""
    m, S, torch, clouds = env
    srv = S.Server(mem_budget_bytes=1 << 30, max_inflight=1, n_streams=1, policy=S.SDF_SERVE_SMALLEST_FIRST,
                   starve_ms=60000)
    cid = srv.register(clouds[1])
    big = torch.as_tensor(f32(synth.uniform_queries(1_000_000, 30)), dtype=torch.float32, device="cuda")
    sizes = [40_000, 5_000, 20_000, 1_000, 10_000]
    xs = [torch.as_tensor(f32(synth.uniform_queries(s, 31 + i)), dtype=torch.float32, device="cuda")
          for i, s in enumerate(sizes)]
    torch.cuda.synchronize()
    outb = torch.empty(big.shape[0], device="cuda")
    tb = srv.submit(S.SDF_REQ_QUERY, cid, big, outb)
    outs = [torch.empty(x.shape[0], device="cuda") for x in xs]
    tk = [srv.submit(S.SDF_REQ_QUERY, cid, x, o) for x, o in zip(xs, outs)]
    srv.poll(tb)
    st = [srv.poll(t) for t in tk]
    order = np.argsort([s["admit_ns"] for s in st])
    assert list(np.array(sizes)[order]) == sorted(sizes)
    for x, o in zip(xs, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), clouds[1].query(x).cpu().numpy())
    srv.shutdown()


def test_express_slot_reserved(env):
    """express_gpairs: with two slots, large requests hold at most one, so
    a small request submitted behind three large ones is admitted before the
    second large one starts, and runs on a high-priority stream; every result
    equals the direct call."""
    m, S, torch, clouds = env
    srv = S.Server(mem_budget_bytes=1 << 30, max_inflight=2, n_streams=2, express_gpairs=1.0)
    cid = srv.register(clouds[1])                      # 20,000 points
    bigs = [torch.as_tensor(f32(synth.uniform_queries(2_000_000, 40 + i)), dtype=torch.float32, device="cuda")
            for i in range(3)]                         # 4e10 pairs each (about 40 ms): bulk
    small = torch.as_tensor(f32(synth.uniform_queries(2_000, 45)), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    outs = [torch.empty(x.shape[0], device="cuda") for x in bigs]
    tb = [srv.submit(S.SDF_REQ_QUERY, cid, x, o) for x, o in zip(bigs, outs)]
    outs_small = torch.empty(small.shape[0], device="cuda")
    ts = srv.submit(S.SDF_REQ_QUERY, cid, small, outs_small)
    st_small = srv.poll(ts)
    st = [srv.poll(t) for t in tb]
    assert st_small["admit_ns"] < st[1]["admit_ns"] and st_small["admit_ns"] < st[2]["admit_ns"]
    assert st[1]["admit_ns"] >= st[0]["done_ns"] - 1_000_000      # one large request at a time
    for x, o in zip(bigs + [small], outs + [outs_small]):
        np.testing.assert_array_equal(o.cpu().numpy(), clouds[1].query(x).cpu().numpy())
    srv.shutdown()


def test_admission_one_slot_in_order(env):
    m, S, torch, clouds = env
    srv = S.Server(mem_budget_bytes=1 << 30, max_inflight=1, n_streams=2)
    cid = srv.register(clouds[1])
    xs = [torch.as_tensor(f32(synth.uniform_queries(5000 + 100 * i, 20 + i)), dtype=torch.float32, device="cuda")
          for i in range(8)]
    outs = [torch.empty(x.shape[0], device="cuda") for x in xs]
    tk = [srv.submit(S.SDF_REQ_QUERY, cid, x, o) for x, o in zip(xs, outs)]
    st = [srv.poll(t) for t in tk]
    for a, b in zip(st, st[1:]):
        assert b["admit_ns"] >= a["done_ns"] - 1_000_000      # one at a time, in arrival order
    for x, o in zip(xs, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), clouds[1].query(x).cpu().numpy())
    srv.shutdown()


def test_refusals_and_timeout(env):
    m, S, torch, clouds = env
    from paper_2607_16946_b300 import SdfError
    srv = S.Server(mem_budget_bytes=1 << 20, max_inflight=2, n_streams=1)
    cid = srv.register(clouds[0])
    x = torch.zeros((200_000, 3), device="cuda")
    out = torch.empty(200_000, device="cuda")
    with pytest.raises(SdfError) as e:
        srv.submit(S.SDF_REQ_QUERY, cid, x, out)          # needs more than the 1 MiB budget
    assert e.value.status == 2
    with pytest.raises(SdfError) as e:
        srv.submit(S.SDF_REQ_QUERY, 99, x[:10], out[:10])
    assert e.value.status == 1
    srv.shutdown()
    srv = S.Server(mem_budget_bytes=4 << 30, max_inflight=2, n_streams=1)
    cid = srv.register(clouds[1])
    big = torch.as_tensor(f32(synth.uniform_queries(2_000_000, 5)), dtype=torch.float32, device="cuda")
    ob = torch.empty(big.shape[0], device="cuda")
    t = srv.submit(S.SDF_REQ_QUERY, cid, big, ob)
    with pytest.raises(TimeoutError):
        srv.poll(t, timeout_s=0.0)
    srv.poll(t)
    srv.shutdown()


def test_weighted_cloud_and_lse_requests(env):
    """A weighted cloud among resident clouds, and log-sum-exp queries: each
    served result equals the direct call bit for bit; the log-sum-exp
    formula is refused for request kinds other than QUERY."""
    m, S, torch, clouds = env
    p, n, a = f32(*synth.ring_torus(6000, 5))
    w = f32(np.exp(np.random.Generator(np.random.PCG64(6)).uniform(-1.0, 1.0, size=len(p))))
    weighted = m.Cloud(p, n, a, weights=w)
    pool = clouds + [weighted]
    srv = S.Server(mem_budget_bytes=2 << 30, max_inflight=4, n_streams=3)
    ids = [srv.register(c) for c in pool]
    rng = np.random.Generator(np.random.PCG64(7))
    cases = []
    for i in range(12):
        ci = int(rng.integers(0, len(pool)))
        kind = S.SDF_REQ_GRAD if i % 4 == 3 else S.SDF_REQ_QUERY
        formula = m.SDF_FORMULA_LSE if (kind == S.SDF_REQ_QUERY and i % 2 == 0) else m.SDF_FORMULA_BLEND
        q = int(rng.integers(500, 40000))
        x = torch.as_tensor(f32(rng.uniform(-1.5, 1.5, size=(q, 3))), dtype=torch.float32, device="cuda")
        out = torch.empty(4 * q if kind == S.SDF_REQ_GRAD else q, device="cuda")
        cases.append((ci, kind, formula, x, out, srv.submit(kind, ids[ci], x, out, formula=formula)))
    for ci, kind, formula, x, out, tk in cases:
        srv.poll(tk)
        if kind == S.SDF_REQ_GRAD:
            phi, g, _ = pool[ci].query_grad(x, saved=False)
            ref = torch.cat([phi, g.reshape(-1)])
        else:
            ref = pool[ci].query(x, formula=formula)
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    x = torch.zeros((10, 3), device="cuda")
    with pytest.raises(m.SdfError):
        srv.submit(S.SDF_REQ_GRAD, ids[0], x, torch.empty(40, device="cuda"), formula=m.SDF_FORMULA_LSE)
    srv.shutdown()
    weighted.close()


def test_large_requests_run_as_chunks_equal_direct(env):
    """Requests above the split budget (split_gpairs) run as query chunks that
    other requests interleave with; each chunk keeps at least one unsplit wave
    of query blocks, so the result equals the direct call bit for bit: a
    device-buffer query, a host-buffer query and a Boolean, submitted with
    small requests in between."""
    m, S, torch, clouds = env
    srv = S.Server(mem_budget_bytes=4 << 30, max_inflight=3, n_streams=3, split_gpairs=1)
    ids = [srv.register(c) for c in clouds]
    rng = np.random.Generator(np.random.PCG64(21))
    q = 2_000_000                                  # 4e10 pairs on the 20,000-point torus
    x = torch.as_tensor(f32(rng.uniform(-1.5, 1.5, size=(q, 3))), dtype=torch.float32, device="cuda")
    xh = x[:1_300_000].cpu().numpy()
    jobs = []
    out = torch.empty(q, device="cuda")
    jobs.append((srv.submit(S.SDF_REQ_QUERY, ids[1], x, out), out, lambda: clouds[1].query(x), 3))
    small_x = [torch.as_tensor(f32(rng.uniform(-1.5, 1.5, size=(2000, 3))), dtype=torch.float32, device="cuda")
               for _ in range(6)]
    for k, sx in enumerate(small_x):
        o = torch.empty(2000, device="cuda")
        jobs.append((srv.submit(S.SDF_REQ_QUERY, ids[k % 4], sx, o), o,
                     (lambda c=clouds[k % 4], sx=sx: c.query(sx)), 1))
    oh = np.empty(xh.shape[0], np.float32)
    jobs.append((srv.submit(S.SDF_REQ_QUERY, ids[1], xh, oh), oh, lambda: clouds[1].query(xh), 2))
    ou = torch.empty(q, device="cuda")
    jobs.append((srv.submit(S.SDF_REQ_UNION, ids[1], x, ou, cloud_id_b=ids[2]), ou,
                 lambda: m.combine(m.SDF_UNION, clouds[1].query(x), clouds[2].query(x)), 3))
    for ticket, o, direct, chunks in jobs:
        st = srv.poll(ticket)
        assert st["chunks"] == chunks
        ref = direct()
        torch.cuda.synchronize()
        got = torch.as_tensor(o) if isinstance(o, np.ndarray) else o.cpu()
        assert torch.equal(got, ref.cpu()), ticket
    srv.shutdown()
