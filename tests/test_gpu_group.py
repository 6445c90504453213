"""GPU: grouped refined Poisson solves (one launch per stage for many boxes).

Every box of a group must give the same bits as the refined solve of its own
plan, alone, and agree with the FP64 CPU oracle to 1e-10 in the relative
max-norm; its result must not depend on the other boxes of the group.
"""

import numpy as np
import pytest

import oracle
from paper_2502_06296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


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
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# boxes of different sizes, stretchings and walls (sizes from the ensemble's
# menus, reduced in z so that the oracle stays quick)
BOXES = [
    (128, 96, 24, 1.2, 0), (64, 48, 32, 2.2, 1), (32, 24, 16, None, 0), (96, 64, 20, 1.8, 0),
    (16, 12, 40, 1.5, 1), (48, 36, 12, 1.6, 0),
]


def make_box(chanfs, i, spec):
    nx, ny, nz, beta, bc = spec
    dz = synth.uniform_dz(nz) if beta is None else synth.tanh_dz(nz, beta)
    f = synth.normal(500 + i, (nz, ny, nx))
    if bc == chanfs.NEUMANN:
        f = synth.remove_weighted_mean(f, dz)
    plan = chanfs.Plan(nx, ny, nz, 12.8, 6.4, dz, bc, chanfs.F32_REFINED)
    return plan, f, dz


def test_group_matches_single_solves_and_oracle(chanfs):
    boxes = [make_box(chanfs, i, s) for i, s in enumerate(BOXES)]
    plans = [b[0] for b in boxes]
    fs = [dev(b[1]) for b in boxes]
    alone = [host(p.poisson_solve(f)) for p, f in zip(plans, fs)]
    alone_info = [p.last_info() for p in plans]
    with chanfs.Group(plans) as g:
        outs = g.poisson_solve(fs)
        info = g.last_info()
        got = [host(o) for o in outs]
        # twice in a row: the group leaves nothing behind
        again = [host(o) for o in g.poisson_solve(fs)]
    for i, (plan, f, dz) in enumerate(boxes):
        nx, ny, nz, beta, bc = BOXES[i]
        assert np.array_equal(got[i], alone[i]), i
        assert np.array_equal(again[i], alone[i]), i
        assert info[i] == alone_info[i], (i, info[i], alone_info[i])
        assert info[i][1] <= TOL and 1 <= info[i][0] <= 4
        ref = oracle.poisson_solve(f, 12.8, 6.4, dz, bc)
        assert rel(got[i], ref) < TOL, (i, rel(got[i], ref))
        assert plan.check() == 0
    for p in plans:
        p.close()


def test_box_result_does_not_depend_on_the_group(chanfs):
    boxes = [make_box(chanfs, i, s) for i, s in enumerate(BOXES)]
    plans = [b[0] for b in boxes]
    fs = [dev(b[1]) for b in boxes]
    with chanfs.Group(plans) as g:
        full = [host(o) for o in g.poisson_solve(fs)]
    with chanfs.Group(plans[2:4]) as g:
        part = [host(o) for o in g.poisson_solve(fs[2:4])]
    with chanfs.Group(plans[::-1]) as g:
        rev = [host(o) for o in g.poisson_solve(fs[::-1])][::-1]
    for i in (2, 3):
        assert np.array_equal(part[i - 2], full[i])
    for i in range(len(plans)):
        assert np.array_equal(rev[i], full[i])
    for p in plans:
        p.close()


def test_group_zero_rhs_and_nonconvergence(chanfs):
    a, fa, _ = make_box(chanfs, 0, (32, 24, 16, 1.5, 0))
    b, fb, _ = make_box(chanfs, 1, (16, 12, 20, 1.8, 1))
    b.set_refinement(1e-14, 1)  # cannot be met with one FP32 solve
    with chanfs.Group([a, b]) as g:
        zero = torch.zeros(16, 24, 32, dtype=torch.float64, device="cuda")
        with pytest.raises(chanfs.ChanfsError) as err:
            g.poisson_solve([zero, dev(fb)])
        assert err.value.status == chanfs.ENOTCONVERGED
        info = g.last_info()
    assert info[0] == (0, 0.0)
    assert info[1][0] == 1 and info[1][1] > 1e-14
    a.close()
    b.close()


def test_group_rejects_bad_arguments(chanfs):
    p64 = chanfs.Plan(16, 12, 10, 1.0, 1.0, np.full(10, 0.2))
    p32 = chanfs.Plan(16, 12, 10, 1.0, 1.0, np.full(10, 0.2), 0, chanfs.F32_REFINED)
    with pytest.raises(chanfs.ChanfsError) as err:
        chanfs.Group([p32, p64])
    assert err.value.status == chanfs.EUNSUPPORTED
    with pytest.raises(chanfs.ChanfsError) as err:
        chanfs.Group([p32, p32])
    assert err.value.status == chanfs.EINVAL
    with chanfs.Group([p32]) as g:
        t = torch.zeros(10, 12, 16, dtype=torch.float64, device="cuda")
        with pytest.raises(chanfs.ChanfsError) as err:
            g.poisson_solve([t], [t])
        assert err.value.status == chanfs.EINVAL
        # fields must start on 16-byte boundaries (rejected before any launch)
        flat = torch.zeros(10 * 12 * 16 + 1, dtype=torch.float64, device="cuda")
        odd = flat[1:].view(10, 12, 16)
        for args in (([odd], [t]), ([t], [odd])):
            with pytest.raises(chanfs.ChanfsError) as err:
                g.poisson_solve(*args)
            assert err.value.status == chanfs.EINVAL
        with pytest.raises(chanfs.ChanfsError) as err:
            g.helmholtz_solve([1e-3], [odd], [0], [t])
        assert err.value.status == chanfs.EINVAL
    p64.close()
    p32.close()


def test_group_helmholtz_matches_single_solves_and_oracle(chanfs):
    boxes = [make_box(chanfs, i, s) for i, s in enumerate(BOXES)]
    plans = [b[0] for b in boxes]
    cs = [1e-6, 3e-5, 1e-4, 9.6e-9, 2e-5, 1e-2]
    locs = [chanfs.CENTER, chanfs.FACE, chanfs.CENTER, chanfs.FACE, chanfs.CENTER, chanfs.FACE]
    rhs = [synth.normal(700 + i, b[1].shape) for i, b in enumerate(boxes)]
    rd = [dev(r) for r in rhs]
    alone = [host(p.helmholtz_solve(c, r, loc)) for p, c, r, loc in zip(plans, cs, rd, locs)]
    alone_info = [p.last_info() for p in plans]
    with chanfs.Group(plans) as g:
        got = [host(o) for o in g.helmholtz_solve(cs, rd, locs)]
        info = g.last_info()
        # a Poisson solve in between does not disturb the next Helmholtz solve
        g.poisson_solve([dev(b[1]) for b in boxes])
        again = [host(o) for o in g.helmholtz_solve(cs, rd, locs)]
    for i, (plan, f, dz) in enumerate(boxes):
        assert np.array_equal(got[i], alone[i]), i
        assert np.array_equal(again[i], alone[i]), i
        assert info[i] == alone_info[i], (i, info[i], alone_info[i])
        ref = oracle.helmholtz_solve(rhs[i], dz, cs[i], locs[i])
        assert rel(got[i], ref) < TOL, (i, rel(got[i], ref))
        assert plan.check() == 0
    for p in plans:
        p.close()


def test_group_ignores_stale_reduction_words(chanfs):
    """A plan's max-norm word may hold anything when a grouped solve starts
    (here: a huge value planted by a refined solve of a large right-hand
    side that was then abandoned); the grouped solve must not read it."""
    plan, f, dz = make_box(chanfs, 0, (32, 24, 16, 1.5, 0))
    x = dev(f)
    alone = host(plan.poisson_solve(x))
    plan.set_refinement(1e-10, 1)
    with pytest.raises(chanfs.ChanfsError):
        plan.poisson_solve(dev(1e30 * f))  # leaves a huge residual norm in the word
    plan.set_refinement(1e-10, 4)
    with chanfs.Group([plan]) as g:
        got = host(g.poisson_solve([x])[0])
        gh = host(g.helmholtz_solve([1e-5], [x])[0])
    assert np.array_equal(got, alone)
    assert np.array_equal(gh, host(plan.helmholtz_solve(1e-5, x)))
    plan.close()


def test_group_helmholtz_with_fp64_direct_boxes(chanfs):
    """Boxes whose plans solve Helmholtz in FP64 directly (CFS_OPT_HELM_FP64)
    run in their own launch of the same group call, bit-identical to their
    single solves, and within 1e-12 of the oracle."""
    boxes = [make_box(chanfs, i, s) for i, s in enumerate(BOXES[:4])]
    plans = [b[0] for b in boxes]
    for p in plans[::2]:
        p.set_option(chanfs.OPT_HELM_FP64, 1)
    cs = [1e-5, 2e-5, 3e-5, 4e-5]
    locs = [chanfs.CENTER, chanfs.FACE, chanfs.FACE, chanfs.CENTER]
    rhs = [synth.normal(800 + i, b[1].shape) for i, b in enumerate(boxes)]
    rd = [dev(r) for r in rhs]
    alone = [host(p.helmholtz_solve(c, r, loc)) for p, c, r, loc in zip(plans, cs, rd, locs)]
    with chanfs.Group(plans) as g:
        got = [host(o) for o in g.helmholtz_solve(cs, rd, locs)]
        info = g.last_info()
    for i, (plan, f, dz) in enumerate(boxes):
        assert np.array_equal(got[i], alone[i]), i
        ref = oracle.helmholtz_solve(rhs[i], dz, cs[i], locs[i])
        assert rel(got[i], ref) < (1e-12 if i % 2 == 0 else TOL), (i, rel(got[i], ref))
        assert (info[i][0] == 0) == (i % 2 == 0), info[i]
        plan.close()


def test_graph_and_host_loop_give_the_same_bits(chanfs):
    """A grouped solve launched as one CUDA graph (refinement loop in a
    conditional node; captured at a launch shape's second solve) and the same
    solve with the loop on the host give identical fields and iteration
    records, for Poisson and for Helmholtz calls of several shapes."""
    boxes = [make_box(chanfs, i, s) for i, s in enumerate(BOXES[:3])]
    plans = [b[0] for b in boxes]
    fs = [dev(b[1]) for b in boxes]
    rhs = [dev(synth.normal(900 + i, b[1].shape)) for i, b in enumerate(boxes)]
    C, F = chanfs.CENTER, chanfs.FACE
    patterns = [[C, C, C], [F, F, F], [C, F, C], [F, C, F], [C, C, F], [F, F, C], [C, C, C]]
    cs = [1e-5, 4e-5, 1e-4]
    with chanfs.Group(plans) as g:
        graph_p = [[host(o) for o in g.poisson_solve(fs)] for _ in range(3)]
        graph_pi = g.last_info()
        graph_h = []
        for locs in patterns:
            for _ in range(2):  # direct launches or a capture, then a graph replay
                graph_h.append(([host(o) for o in g.helmholtz_solve(cs, rhs, locs)],
                                g.last_info()))
        g.set_graphs(False)
        host_p = [host(o) for o in g.poisson_solve(fs)]
        host_pi = g.last_info()
        host_h = []
        for locs in patterns:
            host_h.append(([host(o) for o in g.helmholtz_solve(cs, rhs, locs)], g.last_info()))
    assert graph_pi == host_pi
    for rep in graph_p:
        for a, b in zip(rep, host_p):
            assert np.array_equal(a, b)
    for k, (ga, gi) in enumerate(graph_h):
        ha, hi = host_h[k // 2]
        assert gi == hi
        for a, b in zip(ga, ha):
            assert np.array_equal(a, b)
    for p in plans:
        p.close()


def test_launch_trace(chanfs):
    """Tracing runs a grouped solve as direct launches with an event pair
    around every copy and kernel: the same bits as the graph-launched solve,
    one positive device time per traced operation, and a reset per solve."""
    boxes = [make_box(chanfs, i, s) for i, s in enumerate(BOXES[:3])]
    plans = [b[0] for b in boxes]
    fs = [dev(b[1]) for b in boxes]
    with chanfs.Group(plans) as g:
        ref = [[host(o) for o in g.poisson_solve(fs)] for _ in range(3)][-1]  # graph replay
        info = g.last_info()
        g.set_trace(True)
        got = [host(o) for o in g.poisson_solve(fs)]
        ms = g.trace()
        iters = max(i for i, _ in g.last_info())
        # start copies and kernels, at least one iteration's stages, the tail
        assert len(ms) >= 8 + 6 * iters, (len(ms), iters)
        assert all(t > 0.0 for t in ms) and sum(ms) < 1e3
        assert g.last_info() == info
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        n_p = len(ms)
        g.helmholtz_solve([1e-5] * 3, fs, [chanfs.CENTER] * 3)
        assert 0 < len(g.trace()) < n_p + 40  # counted afresh
        assert g.trace(capacity=2) == g.trace()[:2]
        g.set_trace(False)
        g.poisson_solve(fs)
        assert len(g.trace()) == 0  # untraced solves record nothing
    for p in plans:
        p.close()


def test_rebinding_reuses_or_captures_graphs(chanfs):
    """Rebinding to other boxes (a new launch shape) and back (a cached
    graph, now reading the re-uploaded tables) gives each box its own bits."""
    boxes = [make_box(chanfs, i, s) for i, s in enumerate(BOXES[:4])]
    plans = [b[0] for b in boxes]
    fs = [dev(b[1]) for b in boxes]
    alone = [host(p.poisson_solve(f)) for p, f in zip(plans, fs)]
    with chanfs.Group(plans[:2], capacity=4) as g:
        first = [host(o) for o in g.poisson_solve(fs[:2])]
        g.rebind(plans[1:4])
        second = [host(o) for o in g.poisson_solve(fs[1:4])]
        g.rebind(plans[:2])
        third = [host(o) for o in g.poisson_solve(fs[:2])]
    assert all(np.array_equal(a, b) for a, b in zip(first, alone[:2]))
    assert all(np.array_equal(a, b) for a, b in zip(third, alone[:2]))
    assert all(np.array_equal(a, b) for a, b in zip(second, alone[1:4]))
    for p in plans:
        p.close()


def test_group_helmholtz_with_thomas_boxes(chanfs):
    """Boxes whose Helmholtz systems take Thomas sweeps (FP32 inner solves,
    or FP64 direct) run in their own launches of the same group call,
    bit-identical to their single solves."""
    boxes = [make_box(chanfs, i, s) for i, s in enumerate(BOXES[:4])]
    plans = [b[0] for b in boxes]
    plans[0].set_option(chanfs.OPT_HELM_THOMAS32, 1)
    plans[1].set_option(chanfs.OPT_HELM_FP64, 1)
    plans[1].set_option(chanfs.OPT_HELM_THOMAS, 1)
    plans[2].set_option(chanfs.OPT_HELM_FP64, 1)
    cs = [1e-5, 2e-5, 3e-5, 4e-5]
    locs = [chanfs.FACE, chanfs.CENTER, chanfs.FACE, chanfs.CENTER]
    rhs = [synth.normal(850 + i, b[1].shape) for i, b in enumerate(boxes)]
    rd = [dev(r) for r in rhs]
    alone = [host(p.helmholtz_solve(c, r, loc)) for p, c, r, loc in zip(plans, cs, rd, locs)]
    with chanfs.Group(plans) as g:
        for _ in range(2):  # direct launches, then a captured graph
            got = [host(o) for o in g.helmholtz_solve(cs, rd, locs)]
            for i in range(4):
                assert np.array_equal(got[i], alone[i]), i
    for i, (plan, f, dz) in enumerate(boxes):
        ref = oracle.helmholtz_solve(rhs[i], dz, cs[i], locs[i])
        assert rel(got[i], ref) < (1e-12 if i in (1, 2) else TOL), (i, rel(got[i], ref))
        plan.close()
