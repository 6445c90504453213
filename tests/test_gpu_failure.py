"""GPU: failure detection without a GPU fault.

* Device side: the kernels' bounded waits.  cfs_selftest_wait_timeout runs
  CTAs through the same wait-or-fail helper the TMA-fed kernels use, on a
  barrier that no copy completes (no copy is issued), with a short poll
  limit.  The kernel must return, the failure must reach the plan's status
  word (cfs_plan_check -> CFS_ETIMEOUT) or the caller's, and the plan and the
  device must stay usable: the next solve matches the oracle.
* Host side (the serving loop): a refused plan allocation fails only the
  requests that needed it; a wait that times out leaves its ticket valid; a
  cancelled request completes as cancelled; a server destroyed with requests
  pending finishes them and returns; worker start-ups that fail leave the
  others serving, and a server with none fails at creation.
"""

import ctypes

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


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dtype", [0, 1])
def test_bounded_wait_that_runs_out_is_reported_and_the_plan_goes_on(chanfs, dtype):
    nx, ny, nz = 32, 24, 20
    dz = synth.tanh_dz(nz, 1.5)
    f = synth.remove_weighted_mean(synth.normal(31, (nz, ny, nx)), dz)
    ref = oracle.poisson_solve(f, 2.0, 1.0, dz, 0)
    tol = 1e-12 if dtype == 0 else 1e-10
    with chanfs.Plan(nx, ny, nz, 2.0, 1.0, dz, 0, dtype) as plan:
        assert rel(plan.poisson_solve(torch.from_numpy(f).cuda()).cpu().numpy(), ref) < tol
        assert plan.check() == 0
        rc = chanfs.lib().cfs_selftest_wait_timeout(plan._h, None, 256, _stream())
        assert rc == chanfs.OK
        bits = ctypes.c_int(0)
        assert chanfs.lib().cfs_plan_check(plan._h, ctypes.byref(bits)) == chanfs.ETIMEOUT
        assert bits.value == 1  # the timeout bit alone: no CTA went past its wait
        assert plan.check() == 0  # reported once, then cleared
        p = plan.poisson_solve(torch.from_numpy(f).cuda()).cpu().numpy()
        assert rel(p, ref) < tol
        assert plan.check() == 0


def test_bounded_wait_reports_into_a_caller_status_word(chanfs):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = chanfs.lib().cfs_selftest_wait_timeout(None, ctypes.c_void_p(status.data_ptr()), 64,
                                                _stream())
    assert rc == chanfs.OK
    torch.cuda.synchronize()
    assert int(status.item()) == 1
    # the device still computes: an allocation-free solve reports no failure
    nz, ny, nx = 40, 6, 8
    dz = synth.tanh_dz(nz, 1.4)
    rhs = synth.normal(5, (nz, ny, nx))
    u, st = chanfs.helmholtz_solve_noalloc(dz, 1e-4, torch.from_numpy(rhs).cuda())
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert rel(u.cpu().numpy(), oracle.helmholtz_solve(rhs, dz, 1e-4, 0)) < 1e-12


RUN = (32, 24, 16, 1.6, 0)


def _server(chanfs, **kw):
    srv = chanfs.Server(1 << 30, kw.pop("workers", 2), 8, autotune=False, **kw)
    nx, ny, nz, beta, bc = RUN
    run = srv.add_run(nx, ny, nz, 12.8, 6.4, synth.tanh_dz(nz, beta), bc)
    return srv, run


def _fields(seed):
    nx, ny, nz, beta, _ = RUN
    f = synth.remove_weighted_mean(synth.normal(seed, (nz, ny, nx)), synth.tanh_dz(nz, beta))
    x = torch.from_numpy(f).cuda()
    return f, x, torch.full_like(x, np.nan)


def _poisson_ref(f):
    nx, ny, nz, beta, bc = RUN
    return oracle.poisson_solve(f, 12.8, 6.4, synth.tanh_dz(nz, beta), bc)


@pytest.mark.parametrize("dtype,nbuf", [(0, 2), (1, 10)])
def test_guard_words_around_work_buffers(chanfs, dtype, nbuf):
    """The work buffers kernels write carry guard words: intact after every
    kind of solve (no kernel stores past its buffer), and a byte overwritten
    just before or just after a buffer (a host-side memset into the guard) is
    reported as CFS_EGUARD with the number of damaged buffers."""
    nx, ny, nz = 64, 48, 40
    dz = synth.tanh_dz(nz, 1.6)
    f = synth.remove_weighted_mean(synth.normal(61, (nz, ny, nx)), dz)
    with chanfs.Plan(nx, ny, nz, 2.0, 1.0, dz, 0, dtype) as plan:
        t = torch.from_numpy(f).cuda()
        plan.poisson_solve(t)
        for loc in (chanfs.CENTER, chanfs.FACE):
            plan.helmholtz_solve(1e-4, t, loc)
        plan.helmholtz3d_solve(1e-4, t)
        if dtype == 1:
            plan.set_option(chanfs.OPT_THOMAS_TILE, 1)
            plan.poisson_solve(t)
            with chanfs.Group([plan]) as g:
                g.poisson_solve([t])
                g.helmholtz_solve([1e-4], [t])
        assert plan.check_guards() == 0
        plan.debug_guard_poke(0, False)
        with pytest.raises(chanfs.ChanfsError) as err:
            plan.check_guards()
        assert err.value.status == chanfs.EGUARD
        plan.debug_guard_poke(nbuf - 1, True)
        n = ctypes.c_int(0)
        assert chanfs.lib().cfs_plan_check_guards(plan._h, ctypes.byref(n)) == chanfs.EGUARD
        assert n.value == 2
        with pytest.raises(chanfs.ChanfsError) as err:
            plan.debug_guard_poke(nbuf, False)  # no such buffer
        assert err.value.status == chanfs.EINVAL
        # the plan still solves correctly (the guards are outside its data)
        p = plan.poisson_solve(t).cpu().numpy()
        ref = oracle.poisson_solve(f, 2.0, 1.0, dz, 0)
        assert np.max(np.abs(p - ref)) / np.max(np.abs(ref)) < (1e-12 if dtype == 0 else 1e-10)


def test_refused_plan_allocation_fails_only_its_request(chanfs):
    srv, run = _server(chanfs, workers=1)
    with srv:
        srv.inject_fault(chanfs.FAULT_PLAN_ALLOC, 1)
        f1, x1, o1 = _fields(1)
        status, _ = srv.wait(srv.submit(run, chanfs.REQ_POISSON, x1, o1), 60.0)
        assert status == chanfs.ENOMEM
        f2, x2, o2 = _fields(2)
        status, _ = srv.wait(srv.submit(run, chanfs.REQ_POISSON, x2, o2), 60.0)
        assert status == chanfs.OK
        assert rel(o2.cpu().numpy(), _poisson_ref(f2)) < 1e-10
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 2 and st["plans_created"] == 1


def test_wait_timeout_cancel_and_resume(chanfs):
    srv, run = _server(chanfs)
    with srv:
        srv.pause(True)
        f1, x1, o1 = _fields(3)
        f2, x2, o2 = _fields(4)
        t1 = srv.submit(run, chanfs.REQ_POISSON, x1, o1)
        t2 = srv.submit(run, chanfs.REQ_POISSON, x2, o2)
        with pytest.raises(chanfs.ChanfsError) as err:
            srv.wait(t1, 0.2)  # nothing runs while paused
        assert err.value.status == chanfs.ETIMEOUT
        srv.cancel(t2)
        assert srv.wait(t2, 1.0)[0] == chanfs.ECANCELED
        with pytest.raises(chanfs.ChanfsError):
            srv.cancel(t2)  # retired
        srv.pause(False)
        assert srv.wait(t1, 60.0)[0] == chanfs.OK  # the ticket outlived its timeout
        assert rel(o1.cpu().numpy(), _poisson_ref(f1)) < 1e-10
        assert bool(torch.isnan(o2).all())  # the cancelled request never ran
        st = srv.stats()
        assert st["cancelled"] == 1 and st["failed"] == 0 and st["pending"] == 0


def test_destroy_with_requests_pending_finishes_them(chanfs):
    srv, run = _server(chanfs)
    srv.pause(True)
    work = [_fields(10 + i) for i in range(4)]
    for f, x, o in work:
        srv.submit(run, chanfs.REQ_POISSON, x, o)  # never waited for
    srv.close()  # resumes, finishes the queue, stops
    torch.cuda.synchronize()
    for f, x, o in work:
        assert rel(o.cpu().numpy(), _poisson_ref(f)) < 1e-10


def test_failed_worker_start_ups(chanfs):
    lib = chanfs.lib()
    assert lib.cfs_server_inject_fault(None, chanfs.FAULT_WORKER_START, 2) == chanfs.OK
    srv, run = _server(chanfs, workers=3)  # two of three refused: one serves
    with srv:
        assert srv.stats()["workers_alive"] == 1
        f, x, o = _fields(20)
        assert srv.wait(srv.submit(run, chanfs.REQ_POISSON, x, o), 60.0)[0] == chanfs.OK
        assert rel(o.cpu().numpy(), _poisson_ref(f)) < 1e-10
    assert lib.cfs_server_inject_fault(None, chanfs.FAULT_WORKER_START, 2) == chanfs.OK
    h = ctypes.c_void_p()
    assert lib.cfs_server_create(ctypes.byref(h), 1 << 30, 2, 4, 1, 0) == chanfs.ECUDA
    assert not h.value
    assert lib.cfs_server_inject_fault(None, chanfs.FAULT_WORKER_START, 0) == chanfs.OK
