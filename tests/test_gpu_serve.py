"""GPU: the serving loop (cfs_server_*): continuous batching of Poisson and
Helmholtz requests from several runs, plans resident under a memory budget.

Each result must be bit-identical to the refined solve of the run's plan
alone -- the same in the mix as alone -- and so within 1e-10 of the oracle.
"""

import numpy as np
import pytest

import oracle
from paper_2502_06296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chanfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs as c
    c.lib()
    return c


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


RUNS = [(64, 48, 32, 1.8, 0), (32, 24, 20, 1.4, 1), (96, 64, 16, 2.0, 0), (48, 36, 24, 1.6, 0),
        (16, 12, 40, 1.2, 1)]
HELM = [(9.6e-9, 0), (2e-5, 1), (1e-4, 0)]


def requests(chanfs):
    """A mixed stream: for every run, Poisson and Helmholtz requests."""
    reqs = []
    for k in range(3):
        for r, (nx, ny, nz, beta, bc) in enumerate(RUNS):
            dz = synth.tanh_dz(nz, beta)
            f = synth.normal(1000 + 10 * r + k, (nz, ny, nx))
            if bc == chanfs.NEUMANN:
                f = synth.remove_weighted_mean(f, dz)
            reqs.append((r, chanfs.REQ_POISSON, 0.0, 0, f))
            c, loc = HELM[(r + k) % len(HELM)]
            reqs.append((r, chanfs.REQ_HELMHOLTZ, c, loc, synth.normal(2000 + 10 * r + k, (nz, ny, nx))))
    return reqs


def alone(chanfs, req):
    r, kind, c, loc, f = req
    nx, ny, nz, beta, bc = RUNS[r]
    dz = synth.tanh_dz(nz, beta)
    with chanfs.Plan(nx, ny, nz, 12.8, 6.4, dz, bc, chanfs.F32_REFINED) as plan:
        x = torch.from_numpy(f).cuda()
        out = plan.poisson_solve(x) if kind == chanfs.REQ_POISSON else plan.helmholtz_solve(c, x, loc)
        return host(out)


def serve(chanfs, reqs, budget, workers=3, max_batch=8, slots=1):
    with chanfs.Server(budget, workers, max_batch, autotune=False, slots_per_run=slots) as srv:
        for nx, ny, nz, beta, bc in RUNS:
            srv.add_run(nx, ny, nz, 12.8, 6.4, synth.tanh_dz(nz, beta), bc)
        ins = [torch.from_numpy(q[4]).cuda() for q in reqs]
        outs = [torch.full_like(x, np.nan) for x in ins]
        torch.cuda.synchronize()
        tickets = [srv.submit(q[0], q[1], x, o, q[2], q[3]) for q, x, o in zip(reqs, ins, outs)]
        results = [srv.wait(t, 120.0) for t in tickets]
        stats = srv.stats()
    return [host(o) for o in outs], results, stats


def test_server_results_are_the_same_in_the_mix_as_alone(chanfs):
    reqs = requests(chanfs)
    got, results, stats = serve(chanfs, reqs, budget=8 << 30)
    assert all(s == 0 and lat > 0 for s, lat in results), results
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["max_batch_seen"] > 1  # requests really were batched
    assert stats["plans_created"] == len(RUNS) and stats["plans_evicted"] == 0
    for q, g in zip(reqs, got):
        assert np.array_equal(g, alone(chanfs, q))
    # and the oracle agrees (one request of each kind)
    for q, g in zip(reqs[:2], got[:2]):
        r, kind, c, loc, f = q
        nx, ny, nz, beta, bc = RUNS[r]
        dz = synth.tanh_dz(nz, beta)
        ref = oracle.poisson_solve(f, 12.8, 6.4, dz, bc) if kind == chanfs.REQ_POISSON else \
            oracle.helmholtz_solve(f, dz, c, loc)
        assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) < 1e-10


def test_server_solves_several_requests_of_one_run_at_once(chanfs):
    """With three plan slots per run, requests of the same run are solved in
    one batch (or overlapping batches); every result is still bit-identical to
    the run's plan alone."""
    reqs = [q for q in requests(chanfs) if q[0] in (0, 2)]
    reqs = reqs + [(r, k, c, loc, f[::-1].copy()) for r, k, c, loc, f in reqs]  # more per run
    got, results, stats = serve(chanfs, reqs, budget=8 << 30, workers=2, max_batch=8, slots=3)
    assert all(s == 0 for s, _ in results), results
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["plans_created"] > 2  # more than one plan for a run
    assert stats["plans_resident"] <= 6
    for q, g in zip(reqs, got):
        assert np.array_equal(g, alone(chanfs, q))


def test_server_evicts_plans_under_a_small_budget(chanfs):
    reqs = requests(chanfs)
    # room for about two plans of these sizes at a time
    got, results, stats = serve(chanfs, reqs, budget=6 << 20, workers=2, max_batch=4)
    assert all(s == 0 for s, _ in results)
    assert stats["plans_evicted"] > 0 and stats["plans_created"] > len(RUNS)
    assert stats["bytes_in_use"] <= 6 << 20
    for q, g in zip(reqs[::5], got[::5]):
        assert np.array_equal(g, alone(chanfs, q))


def test_server_rejects_bad_requests(chanfs):
    with chanfs.Server(1 << 30, 1, 4, autotune=False) as srv:
        with pytest.raises(chanfs.ChanfsError) as err:
            srv.add_run(1024, 1024, 1024, 1.0, 1.0, np.full(1024, 1e-3))  # plan alone > budget
        assert err.value.status == chanfs.EUNSUPPORTED
        run = srv.add_run(16, 12, 10, 1.0, 1.0, np.full(10, 0.2))
        x = torch.zeros(10, 12, 16, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        lib = chanfs.lib()
        import ctypes
        t = ctypes.c_ulonglong(0)
        px, py = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())
        assert lib.cfs_server_submit(srv._h, 5, 0, 0.0, 0, px, py, ctypes.byref(t)) == chanfs.EINVAL
        assert lib.cfs_server_submit(srv._h, run, 1, 1e-5, 7, px, py, ctypes.byref(t)) == chanfs.EINVAL
        assert lib.cfs_server_submit(srv._h, run, 0, 0.0, 0, px, px, ctypes.byref(t)) == chanfs.EINVAL
        assert lib.cfs_server_submit(srv._h, run, 3, 0.0, 0, px, py, ctypes.byref(t)) == chanfs.EINVAL
        assert lib.cfs_server_cancel(srv._h, 987654) == chanfs.EINVAL
        assert lib.cfs_server_inject_fault(srv._h, 99, 1) == chanfs.EINVAL
        assert lib.cfs_server_inject_fault(srv._h, chanfs.FAULT_WORKER_START, 1) == chanfs.EINVAL
        ticket = srv.submit(run, chanfs.REQ_POISSON, x, y)
        assert srv.wait(ticket, 60.0)[0] == 0
        assert np.all(host(y) == 0.0)  # zero right-hand side
