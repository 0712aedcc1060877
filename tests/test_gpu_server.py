"""Serving loop: requests of mixed size, omega, time grid and precision
submitted while others run; each result must match the oracle, and must be
identical whether the request ran alone or in the mix."""
import threading
import time

import numpy as np
import pytest

from oracle import expmv, graph, superop
from paper_2003_02450_gb300 import workloads as W
from tests.libbuild import ensure_built

pytestmark = pytest.mark.gpu


def _requests(count, seed):
    from paper_2003_02450_gb300 import qsw as C
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(count):
        n = int(round(np.exp(rng.uniform(np.log(6), np.log(48)))))
        g = W.erdos_renyi_mean_degree(n, 3.0, seed * 1000 + k)
        omega = float(rng.uniform(0, 1))
        steps = int(rng.integers(1, 40))
        prec = "c64" if k % 2 else "c128"
        t0 = float(rng.choice([0.0, 0.3]))
        if k % 3 == 0:
            r = C.Request(g, omega, t0, 0.1, steps, prec, populations=np.eye(n)[0])
            rho0 = W.basis_state(n, 0)
        else:
            rho0 = W.random_pure_states(n, 1, seed * 1000 + k)[0]
            r = C.Request(g, omega, t0, 0.1, steps, prec, rho0=rho0)
        r.meta = (g, omega, rho0, t0, steps, prec)
        reqs.append(r)
    return reqs


def _oracle_pops(g, omega, rho0, t0, steps):
    walk = graph.lqsw_walk(graph.adjacency(g))
    L = superop.superoperator(walk, omega)
    X = expmv.expmv_series(L, W.vec(rho0), t0, 0.1, steps)
    return superop.populations(X, walk.n_tilde)


def test_server_mix_matches_oracle_and_alone():
    ensure_built()
    from paper_2003_02450_gb300 import qsw as C
    reqs = _requests(24, 3)
    srv = C.qsw_server_create(0, workers=3, max_batch=8, memory_budget_bytes=64e6)
    try:
        # submit from two threads, staggered, so that batches overlap
        def submit(part):
            for r in part:
                C.qsw_server_submit(srv, r)
                time.sleep(0.002)
        ths = [threading.Thread(target=submit, args=(reqs[i::2],)) for i in range(2)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        res = [C.qsw_server_wait(srv, r, 300.0) for r in reqs]
        st = C.qsw_server_stats(srv)
    finally:
        C.qsw_server_destroy(srv)
    assert st["batches"] >= 2 and st["queued"] == 0
    for r, info in zip(reqs, res):
        g, omega, rho0, t0, steps, prec = r.meta
        ref = _oracle_pops(g, omega, rho0, t0, steps)
        tol = 1e-10 if prec == "c128" else 1e-4
        assert np.max(np.abs(r.pops - ref)) <= tol
        assert info["latency_ms"] >= info["queue_ms"] >= 0.0
    # alone: the same request through a fresh server, one at a time
    srv = C.qsw_server_create(0, workers=1, max_batch=1)
    try:
        for r in reqs:
            g, omega, rho0, t0, steps, prec = r.meta
            alone = C.Request(g, omega, t0, 0.1, steps, prec, rho0=rho0)
            C.qsw_server_submit(srv, alone)
            C.qsw_server_wait(srv, alone, 300.0)
            assert np.array_equal(alone.pops, r.pops)      # bit-identical alone and in the mix
    finally:
        C.qsw_server_destroy(srv)


def test_server_isolates_bad_requests_and_oversized_ones():
    ensure_built()
    from paper_2003_02450_gb300 import qsw as C
    good = _requests(3, 9)
    loop = W.Digraph(3, np.array([0, 1, 1, 1], np.int32), np.array([0], np.int32), np.array([1.0]))
    bad = C.Request(loop, 0.5, 0.0, 0.1, 3, "c128", populations=[1.0, 0, 0])
    big = _requests(1, 11)[0]
    srv = C.qsw_server_create(0, workers=2, max_batch=4, memory_budget_bytes=1.0)  # everything oversized
    try:
        for r in good + [bad, big]:
            C.qsw_server_submit(srv, r)
        for r in good + [big]:
            C.qsw_server_wait(srv, r, 300.0)
        with pytest.raises(C.QswError) as e:
            C.qsw_server_wait(srv, bad, 300.0)
        assert e.value.name == "QSW_ERR_NOT_SIMPLE"
    finally:
        C.qsw_server_destroy(srv)
    for r in good + [big]:
        g, omega, rho0, t0, steps, prec = r.meta
        tol = 1e-10 if prec == "c128" else 1e-4
        assert np.max(np.abs(r.pops - _oracle_pops(g, omega, rho0, t0, steps))) <= tol


def test_server_concurrent_small_batches_of_mixed_sizes():
    """Many small walks of different sizes through 4 workers with small batches:
    concurrent batched launches with different shared-memory sizes must all
    succeed (the small-walk kernel's limit is shared by every stream) and match
    the oracle on a sample."""
    ensure_built()
    from paper_2003_02450_gb300 import qsw as C
    rng = np.random.default_rng(12)
    reqs = []
    for k in range(96):
        n = int(rng.choice([6, 11, 17, 24, 31, 40]))
        g = W.erdos_renyi_mean_degree(n, 3.0, 7000 + k)
        prec = "c64" if k % 2 else "c128"
        r = C.Request(g, 0.4, 0.0, 0.1, int(rng.integers(2, 30)), prec, populations=np.eye(n)[0])
        r.meta = (g, 0.4, W.basis_state(n, 0), 0.0, prec)
        reqs.append(r)
    srv = C.qsw_server_create(0, workers=4, max_batch=3, memory_budget_bytes=256e6)
    try:
        for r in reqs:
            C.qsw_server_submit(srv, r)
        for r in reqs:
            C.qsw_server_wait(srv, r, 300.0)
    finally:
        C.qsw_server_destroy(srv)
    for r in reqs[:6]:
        g, omega, rho0, t0, prec = r.meta
        ref = _oracle_pops(g, omega, rho0, t0, r.c.steps)
        tol = 1e-10 if prec == "c128" else 1e-4
        assert np.max(np.abs(r.pops - ref)) <= tol


def _big_requests(seed):
    """Config-5-style walks that take the whole-GPU series kernel (N >= 160):
    directed Erdos-Renyi graphs of mean out-degree 8, w ~ U(0.5, 1.5), each
    graph served once in complex128 and once in complex64 bulk."""
    from paper_2003_02450_gb300 import qsw as C
    rng = np.random.default_rng(seed)
    reqs = []
    for k, n in enumerate((160, 300, 600)):
        g = W.erdos_renyi_mean_degree(n, 8.0, seed * 100 + k)
        omega = float(rng.uniform(0, 1))
        steps = int(rng.integers(5, 25))
        rho0 = W.random_pure_states(n, 1, seed * 100 + k)[0] if k % 2 else W.basis_state(n, 0)
        for prec in ("c128", "c64"):
            if k % 2:
                r = C.Request(g, omega, 0.0, 0.1, steps, prec, rho0=rho0)
            else:
                r = C.Request(g, omega, 0.0, 0.1, steps, prec, populations=np.eye(n)[0])
            r.meta = (g, omega, rho0, 0.0, steps, prec)
            r.key = k
            reqs.append(r)
    return reqs


def test_server_mix_with_whole_gpu_walks_matches_oracle_and_alone():
    """Whole-GPU walks (cooperative series kernel on one worker's stream) run
    beside batched small walks on the other workers' streams.  Every result
    matches the oracle and is bit-identical to the same request served alone."""
    ensure_built()
    from paper_2003_02450_gb300 import qsw as C
    small = _requests(18, 21)
    big = _big_requests(31)
    mix = []
    for k in range(max(len(small), len(big))):   # interleave: big ones arrive among small ones
        if k < len(big):
            mix.append(big[k])
        if k < len(small):
            mix.append(small[k])
    srv = C.qsw_server_create(0, workers=3, max_batch=6, memory_budget_bytes=4e9)
    try:
        def submit(part):
            for r in part:
                C.qsw_server_submit(srv, r)
                time.sleep(0.003)
        ths = [threading.Thread(target=submit, args=(mix[i::3],)) for i in range(3)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for r in mix:
            C.qsw_server_wait(srv, r, 600.0)
        st = C.qsw_server_stats(srv)
    finally:
        C.qsw_server_destroy(srv)
    assert st["queued"] == 0 and st["batches"] >= 4
    # oracle: one FP64 series per distinct walk (the c128 / c64 pair of a big graph share it)
    refs = {}
    for r in mix:
        g, omega, rho0, t0, steps, prec = r.meta
        key = ("big", r.key) if hasattr(r, "key") else ("small", id(r))
        if key not in refs:
            refs[key] = _oracle_pops(g, omega, rho0, t0, steps)
        tol = 1e-10 if prec == "c128" else 1e-4
        err = np.max(np.abs(r.pops - refs[key]))
        assert err <= tol, (g.n, prec, err)
    # alone: each request through a fresh one-worker server, one at a time
    srv = C.qsw_server_create(0, workers=1, max_batch=1)
    try:
        for r in mix:
            g, omega, rho0, t0, steps, prec = r.meta
            alone = C.Request(g, omega, t0, 0.1, steps, prec, rho0=rho0)
            C.qsw_server_submit(srv, alone)
            C.qsw_server_wait(srv, alone, 600.0)
            assert np.array_equal(alone.pops, r.pops), (g.n, prec)
    finally:
        C.qsw_server_destroy(srv)


def test_server_completes_short_walks_of_a_batch_first():
    """One batched launch holding one long walk (N = 120, 100 steps) and
    several tiny ones (N = 6..10, 2 steps): each walk's result is handed out as
    soon as its cluster has finished it, so the tiny walks complete (and their
    latency is measured) well before the long one; results match the oracle."""
    ensure_built()
    from paper_2003_02450_gb300 import qsw as C
    big_g = W.erdos_renyi_mean_degree(120, 8.0, 4242)
    big = C.Request(big_g, 0.4, 0.0, 0.1, 100, "c128", populations=np.eye(120)[0])
    small = []
    for k in range(6):
        n = 6 + k % 5
        g = W.erdos_renyi_mean_degree(n, 3.0, 500 + k)
        r = C.Request(g, 0.5, 0.0, 0.1, 2, "c128", populations=np.eye(n)[0])
        r.meta = (g, n)
        small.append(r)
    # one worker, one batch: the long walk is submitted first, the tiny ones
    # right behind it, so that the worker takes all of them into one launch
    srv = C.qsw_server_create(0, workers=1, max_batch=16, memory_budget_bytes=4e9)
    try:
        # a whole-GPU walk (N >= 160 runs alone) keeps the only worker busy
        # while the seven walks queue up behind it; the worker then takes all
        # seven into one batched launch
        blocker = C.Request(W.erdos_renyi_mean_degree(300, 8.0, 77), 0.3, 0.0, 0.1, 60, "c128",
                            populations=np.eye(300)[0])
        C.qsw_server_submit(srv, blocker)
        for r in [big] + small:
            C.qsw_server_submit(srv, r)
        C.qsw_server_wait(srv, blocker, 300.0)
        res_big = C.qsw_server_wait(srv, big, 300.0)
        res_small = [C.qsw_server_wait(srv, r, 300.0) for r in small]
        st = C.qsw_server_stats(srv)
    finally:
        C.qsw_server_destroy(srv)
    assert st["batches"] == 2, st   # the blocker, then one launch holding all seven
    assert max(x["latency_ms"] for x in res_small) < res_big["latency_ms"]
    for r in small:
        g, n = r.meta
        ref = _oracle_pops(g, 0.5, W.basis_state(n, 0), 0.0, 2)
        assert np.max(np.abs(r.pops - ref)) <= 1e-10
    ref = _oracle_pops(big_g, 0.4, W.basis_state(120, 0), 0.0, 100)
    assert np.max(np.abs(big.pops - ref)) <= 1e-10
