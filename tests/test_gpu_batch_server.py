"""Batched solves and the request server: every result equals the same
problem solved alone (bitwise: fixed reduction orders, kernel choice cached
per shape, and a packed sweep's arithmetic per subdomain does not depend on
what else is in the launch), admission against the HBM budget, error paths."""

import time

import numpy as np
import pytest

from workloads import configs

pytestmark = pytest.mark.gpu


def _mix():
    base = configs.config1()
    return [
        configs.Workload("mixA", (0, 1, 0, 1), 16, 16, 2, 4, 4, 9.0, "const", (0.3, 0.6), 0.05),
        configs.Workload("mixB", (0, 1, 0, 1), 12, 12, 3, 4, 4, 14.0, "channel", (0.5, 0.3), 0.03),
        configs.Workload("mixC", (0, 1, 0, 1), 8, 16, 4, 4, 8, 6.0, "random", (0.4, 0.5), 0.05, corr_len=0.3),
        configs.scaled(base, 16, 16, 8, 8, name="mixD"),
    ]


def _opts(hz, pack=1):
    return hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=1e-8, pack=pack)


def test_batch_equals_individual_solves(hz):
    """Unpacked batch: each solve launches its own (autotuned) sweeps, so
    the results equal the solo solves bitwise."""
    from paper_2606_21695_gb300.api import Case

    cases = [Case(wl) for wl in _mix()]
    solo = []
    for c in cases:
        st, u, rep = hz.hz_solve(c.pr, _opts(hz), n=c.n)
        assert st == hz.HZ_OK, rep
        assert rep["sweep_variant"] in (1, 2, 3)
        solo.append(u.copy())
    st, sts, us, reps = hz.hz_solve_batch([c.pr for c in cases], [c.n for c in cases], _opts(hz, pack=0),
                                          max_concurrent=4)
    assert st == hz.HZ_OK and all(s == hz.HZ_OK for s in sts)
    for k in range(len(cases)):
        assert reps[k]["rel_residual"] <= 1e-8
        assert np.array_equal(us[k], solo[k]), k


def test_packed_batch_same_alone_and_in_mix(hz):
    """Packed batch: one launch per outer step sweeps every member; a
    problem's result is bitwise the same batched alone or with the others,
    and within the solve tolerance of the unpacked solve."""
    from paper_2606_21695_gb300.api import Case

    cases = [Case(wl) for wl in _mix()]
    packable = [0, 1, 3]  # (P, sub_ny) = (2, 4), (3, 4), (2, 8); mixC has (4, 8): unpacked
    alone = []
    for c in cases:
        st, sts, us, reps = hz.hz_solve_batch([c.pr], [c.n], _opts(hz))
        assert st == hz.HZ_OK
        alone.append((us[0].copy(), reps[0]))
    for k, (u, rep) in enumerate(alone):
        assert rep["rel_residual"] <= 1e-8
        assert rep["sweep_variant"] == 4 if k in packable else rep["sweep_variant"] in (1, 2, 3)
    for order in ([0, 1, 2, 3], [3, 2, 1, 0]):
        sub = [cases[k] for k in order]
        st, sts, us, reps = hz.hz_solve_batch([c.pr for c in sub], [c.n for c in sub], _opts(hz))
        assert st == hz.HZ_OK and all(s == hz.HZ_OK for s in sts)
        for i, k in enumerate(order):
            assert np.array_equal(us[i], alone[k][0]), k
            assert reps[i]["sweeps"] == alone[k][1]["sweeps"]
    for k in packable:
        st, u, rep = hz.hz_solve(cases[k].pr, _opts(hz), n=cases[k].n)
        # both solves stop at a relative residual of 1e-8
        assert np.max(np.abs(alone[k][0] - u)) <= 1e-5 * np.max(np.abs(u))


def test_server_results_same_alone_and_in_mix(hz):
    from paper_2606_21695_gb300.api import Case

    cases = [Case(wl) for wl in _mix()]
    srv = hz.hz_server_create(0, 8 << 30)
    try:
        solo = []
        for c in cases:  # each request served alone
            done, st, u, rep = hz.hz_server_poll(srv, hz.hz_server_submit(srv, c.pr, _opts(hz)), -1, n=c.n)
            assert done and st == hz.HZ_OK and rep["rel_residual"] <= 1e-8
            solo.append(u.copy())
        tickets = []
        for rnd in range(2):  # requests arrive while others run
            for c in cases:
                tickets.append((hz.hz_server_submit(srv, c.pr, _opts(hz)), c))
            time.sleep(0.01)
        for t, c in tickets:
            done, st, u, rep = hz.hz_server_poll(srv, t, -1, n=c.n)
            assert done and st == hz.HZ_OK
            k = cases.index(c)
            assert np.array_equal(u, solo[k])
        stats = hz.hz_server_stats(srv)
        assert stats["p99_ms"] >= stats["p50_ms"] > 0 and stats["solves_per_s"] > 0
        assert stats["hbm_in_use"] == 0
        with pytest.raises(hz.HzError) as e:
            hz.hz_server_poll(srv, 987654, 0, n=cases[0].n)
        assert e.value.status == hz.HZ_ERR_NOT_FOUND
    finally:
        hz.hz_server_destroy(srv)


def test_server_admission_refuses_over_budget_without_disturbing_others(hz):
    from paper_2606_21695_gb300.api import Case

    small = Case(_mix()[0])  # 1089 nodes, 16 subdomains: about 2 MiB of device state
    big = Case(configs.scaled(configs.config2(), 128, 128, 8, 8, name="big"))  # 148k nodes, 256 subdomains: ~40 MiB
    srv = hz.hz_server_create(0, 16 << 20)  # 16 MiB: the small problem fits, the big one does not
    try:
        t = hz.hz_server_submit(srv, small.pr, _opts(hz))
        with pytest.raises(hz.HzError) as e:
            hz.hz_server_submit(srv, big.pr, _opts(hz))
        assert e.value.status == hz.HZ_ERR_BUSY
        done, st, u, rep = hz.hz_server_poll(srv, t, -1, n=small.n)
        assert done and st == hz.HZ_OK and rep["rel_residual"] <= 1e-8
        # a poll with zero timeout on an unfinished request reports not done
        t2 = hz.hz_server_submit(srv, small.pr, _opts(hz))
        done0, _, _, _ = hz.hz_server_poll(srv, t2, 0, n=small.n)
        done1, st1, _, _ = hz.hz_server_poll(srv, t2, -1, n=small.n)
        assert done1 and st1 == hz.HZ_OK
    finally:
        hz.hz_server_destroy(srv)


def test_server_queued_requests_hold_no_device_memory(hz):
    """A burst larger than the HBM budget: queued requests are host
    snapshots, so the device memory the server holds stays within the budget
    it admits against (plus the per-solve allocations the estimate covers
    loosely), and the admitted bytes never exceed the budget.  The solves are
    cut short (40 sweeps): only their memory matters here."""
    import torch

    from paper_2606_21695_gb300.api import Case

    big = Case(configs.scaled(configs.config2(), 128, 128, 8, 8, name="burst"))  # 148k nodes, 256 subdomains
    opts = hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=1e-8, max_sweeps=40)
    ok = (hz.HZ_OK, hz.HZ_ERR_NOT_CONVERGED)
    srv = hz.hz_server_create(0, 96 << 20)  # about two such solves at a time
    try:
        # one request first, so module loading and the first solve's tuning are not counted
        done, st, _, _ = hz.hz_server_poll(srv, hz.hz_server_submit(srv, big.pr, opts), -1, n=big.n)
        assert done and st in ok
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        n_req = 48  # their fields alone (c, f: 24 bytes per node) would be ~170 MB on the device
        tickets = [hz.hz_server_submit(srv, big.pr, opts) for _ in range(n_req)]
        peak = 0
        for _ in range(40):
            free, _ = torch.cuda.mem_get_info()
            peak = max(peak, free0 - free)
            assert hz.hz_server_stats(srv)["hbm_in_use"] <= 96 << 20
            time.sleep(0.01)
        print("burst: device bytes held above the idle level", peak)
        assert peak <= (96 << 20) + (64 << 20)
        for t in tickets:
            done, st, _, _ = hz.hz_server_poll(srv, t, -1, n=big.n)
            assert done and st in ok
        assert hz.hz_server_stats(srv)["hbm_in_use"] == 0
    finally:
        hz.hz_server_destroy(srv)
        big.close()
