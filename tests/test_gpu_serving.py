"""a9 on the GPU: the request loop (continuous batching with memory
admission) through ed_server_* / ed_submit / ed_poll.

* a request gives the same result alone and inside a mix of other requests
  (bit for bit: the kernels and reductions are deterministic and requests
  share no data), and the same as the direct ed_solve call;
* requests that arrive while another runs are admitted and overlap with it;
* admission by device memory: a request larger than the budget is refused at
  submit, and a budget that fits one request at a time serialises them;
* failures are injected on the host (an allocation failure) and reported per
  request; ed_poll never blocks and ed_wait times out."""
import time

import numpy as np
import pytest

from oracle import fock, lanczos
from workloads import make_model, serving_stream

pytestmark = pytest.mark.gpu

OPTS = dict(precision="fp32_polish", gf_precision="fp32", nmats=64, beta=50.0, gf_steps=60)


def _req_models(n, seed=3, max_ns=10):
    return [q.workload for q in serving_stream(n, rate_per_s=1e9, seed=seed, max_ns=max_ns)]


def _wait_all(srv, tickets, timeout=300.0):
    out = {}
    for t in tickets:
        assert srv.wait(t, timeout) == 0
        r = srv.poll(t)
        assert r is not None
        out[t] = r
    return out


def test_same_result_alone_in_mix_and_direct(ed):
    wls = _req_models(12)
    target = wls[5]
    with ed.Server(slots=6) as srv:
        t_alone = srv.submit(target.model, target.nup, target.ndw, **OPTS)
        alone = _wait_all(srv, [t_alone])[t_alone]
        mix = [srv.submit(w.model, w.nup, w.ndw, **OPTS) for w in wls]
        res = _wait_all(srv, mix)
    in_mix = res[mix[5]]
    assert alone[0]["status"] == 0 and in_mix[0]["status"] == 0
    assert alone[0]["e0"] == in_mix[0]["e0"]
    assert np.array_equal(alone[1], in_mix[1])
    direct, G = ed.solve(target.model, target.nup, target.ndw, **OPTS)
    assert direct["e0"] == alone[0]["e0"]
    assert np.array_equal(G, alone[1])
    # every request of the mix against the FP64 oracle energy (small sectors)
    for w, t in zip(wls, mix):
        s = fock.Sector(w.model, w.nup, w.ndw)
        if s.dim > 40000:
            continue
        ro = lanczos.lanczos_ground(s.matvec, lanczos.start_vector(0x5EED, s.dim))
        assert abs(res[t][0]["e0"] - ro["e0"]) <= 1e-9 * max(1, abs(ro["e0"]))


def test_requests_overlap_and_complete_out_of_order(ed):
    big = make_model(2, 6, U=3.0, Jh=0.5, seed=9)          # Ns=14, (7,7): D = 11.8M
    small = _req_models(6, seed=5, max_ns=8)
    big_opts = dict(OPTS, gf_steps=200, nmats=512)
    with ed.Server(slots=4) as srv:
        tb = srv.submit(big, 7, 7, **big_opts)
        time.sleep(0.02)                                    # arrive while the big one runs
        ts = [srv.submit(w.model, w.nup, w.ndw, **OPTS) for w in small]
        res = _wait_all(srv, [tb] + ts)
    rb = res[tb][0]
    assert rb["status"] == 0
    assert all(res[t][0]["status"] == 0 for t in ts)
    # the three free slots take small requests while the big one runs
    started = sorted(res[t][0]["t_start_s"] for t in ts)
    assert started[2] < rb["t_done_s"]
    assert min(res[t][0]["t_done_s"] for t in ts) < rb["t_done_s"]


def test_memory_admission(ed):
    wls = _req_models(4, seed=7, max_ns=8)
    # a budget below every request's estimate: refused at submit
    with ed.Server(slots=2, device_mem_budget=1 << 20) as srv:
        with pytest.raises(ed.EDError) as e:
            srv.submit(wls[0].model, wls[0].nup, wls[0].ndw, **OPTS)
        assert e.value.status == ed.ED_ERR_OOM
    # a budget that fits one request at a time: no two run together
    with ed.Server(slots=4, device_mem_budget=40 << 20) as srv:
        ts = [srv.submit(w.model, w.nup, w.ndw, **OPTS) for w in wls]
        res = _wait_all(srv, ts)
    spans = sorted((r[0]["t_start_s"], r[0]["t_done_s"]) for r in res.values())
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-6


def test_injected_allocation_failure_and_polling(ed):
    wls = _req_models(3, seed=11, max_ns=8)
    with ed.Server(slots=1) as srv:
        srv.inject_alloc_failure(1)
        ts = [srv.submit(w.model, w.nup, w.ndw, **OPTS) for w in wls]
        first = srv.poll(ts[-1])                            # never blocks
        assert first is None or first[0]["status"] in (0, ed.ED_ERR_OOM)
        res = _wait_all(srv, ts if first is None else ts[:-1])
        if first is not None:
            res[ts[-1]] = first
        assert res[ts[0]][0]["status"] == ed.ED_ERR_OOM
        assert res[ts[1]][0]["status"] == 0 and res[ts[2]][0]["status"] == 0
        with pytest.raises(ed.EDError) as e:
            srv.poll(123456789)
        assert e.value.status == ed.ED_ERR_NOT_FOUND
        big = make_model(2, 6, U=3.0, Jh=0.5, seed=9)
        t = srv.submit(big, 7, 7, **OPTS)
        assert srv.wait(t, 0.001) == ed.ED_ERR_TIMEOUT      # bounded wait
        assert srv.wait(t, 300.0) == 0


def test_small_requests_share_chain_launches(ed):
    """Requests whose Green's-function chains live in small sectors (every
    N+-1 sector at most 2^14 states: Ns=8 and Norb=2 Ns=8 sectors here) and
    that reach that phase together share one persistent launch of their
    chains (ed_batch_stats counts launches that merged several solves); every
    request's E0 and G are the same, bit for bit, as the same request solved
    alone in a launch of its own."""
    rng = np.random.default_rng(8)
    reqs = []
    for i in range(24):
        if i % 2:
            m = make_model(1, 7, U=float(rng.uniform(1, 4)), seed=100 + i)
            nup, ndw = 4 + (i % 3 == 0), 4
        else:
            m = make_model(2, 3, U=float(rng.uniform(1, 4)), Jh=0.3, seed=200 + i)
            nup, ndw = 4, 4 - (i % 4 == 0)
        reqs.append((m, nup, ndw))
    alone = [ed.solve(m, nup, ndw, **OPTS) for (m, nup, ndw) in reqs]
    before = ed.batch_stats()
    with ed.Server(slots=8) as srv:
        tickets = [srv.submit(m, nup, ndw, **OPTS) for (m, nup, ndw) in reqs]
        res = _wait_all(srv, tickets)
    after = ed.batch_stats()
    # every request's chains ran batched, and some launches merged solves:
    # fewer launches than requests
    assert 0 < after["launches"] - before["launches"] < len(reqs)
    assert after["max_solves"] >= 2
    for (r_alone, G_alone), t in zip(alone, tickets):
        r_mix, G_mix = res[t]
        assert r_mix["status"] == 0
        assert r_mix["e0"] == r_alone["e0"]
        assert np.array_equal(G_mix, G_alone)
