"""GPU: a seeded sweep over many small plan shapes against the oracle.

Each case draws a grid (x and y lengths with prime factors 2 and 3 only, as
the transforms require; 3..80 cells in z, uniform or tanh-stretched), the
wall conditions (z: Neumann or Dirichlet; y: periodic, Neumann or Dirichlet
walls), the precision (FP64, or FP32 solves with FP64 refinement) and kernel
shapes (z-solve kernel, Algorithm 2 partitions, Thomas or Algorithm 2 for
Helmholtz), then checks a Poisson and a Helmholtz solve (and for some a
fully implicit Helmholtz solve) element by element against the oracle:
relative max-norm 1e-12 for FP64 plans, 1e-10 for refined ones; the
host-buffer and stage-by-stage entry points must give the solve's bits.  Shapes the library declines (CFS_EUNSUPPORTED) are skipped
and counted; most must be accepted.
"""

import numpy as np
import pytest

import oracle
from paper_2502_06296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

def _smooth(n):
    """True when n has no prime factors other than 2 and 3."""
    for p in (2, 3):
        while n % p == 0:
            n //= p
    return n == 1


SMOOTH = [n for n in range(1, 97) if _smooth(n)]


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


def draw(rng, chanfs):
    refined = bool(rng.integers(2))
    while True:
        m = int(rng.choice([k for k in SMOOTH if 2 <= k <= 48]))
        nx = 2 * m
        if not refined or nx % 4 == 0:
            break
    ny = int(rng.choice([k for k in SMOOTH if k <= 96]))
    nz = int(rng.integers(4, 81))
    beta = float(rng.choice([0.0, 1.2, 1.8, 2.4]))
    bc = int(rng.integers(2))
    ybc = int(rng.choice([0, 0, 1, 2]))
    c = float(10.0 ** rng.uniform(-6, -2))
    loc = int(rng.integers(2))
    opts = {"thomas": int(rng.choice([0, -1, 8, 16] + ([1] if refined else []))),
            "parts": int(rng.choice([0, 0, 2, 4, 8])),
            "helm_thomas": int(rng.integers(2)),
            "helm_fp64": int(rng.integers(2)) if refined else 0,
            "helm_thomas32": int(rng.integers(2)) if refined else 0}
    return dict(refined=refined, nx=nx, ny=ny, nz=nz, beta=beta, bc=bc, ybc=ybc, c=c, loc=loc,
                opts=opts)


def test_random_plans_match_the_oracle(chanfs):
    rng = np.random.default_rng(2502)
    ran = skipped = 0
    for case in range(96):
        d = draw(rng, chanfs)
        nx, ny, nz = d["nx"], d["ny"], d["nz"]
        lx, ly = 2.0 + nx / 64.0, 1.0 + ny / 64.0
        dz = synth.uniform_dz(nz) if d["beta"] == 0.0 else synth.tanh_dz(nz, d["beta"])
        dtype = chanfs.F32_REFINED if d["refined"] else chanfs.F64
        try:
            plan = chanfs.Plan(nx, ny, nz, lx, ly, dz, d["bc"], dtype, d["ybc"])
        except chanfs.ChanfsError as e:
            assert e.status == chanfs.EUNSUPPORTED, (d, e)
            skipped += 1
            continue
        with plan:
            for opt, key in ((chanfs.OPT_THOMAS_TILE, "thomas"), (chanfs.OPT_PCR_PARTS, "parts"),
                             (chanfs.OPT_HELM_THOMAS, "helm_thomas")):
                try:
                    plan.set_option(opt, d["opts"][key])
                except chanfs.ChanfsError as e:
                    assert e.status == chanfs.EUNSUPPORTED, (d, key, e)
            tol = 1e-10 if d["refined"] else 1e-12
            f = synth.normal(1000 + case, (nz, ny, nx))
            if d["bc"] == 0 and d["ybc"] != 2:  # the constants are the null space
                f = synth.remove_weighted_mean(f, dz)
            ref = (oracle.poisson_solve(f, lx, ly, dz, d["bc"]) if d["ybc"] == 0 else
                   oracle.poisson_solve_walls(f, lx, ly, dz, d["bc"], d["ybc"]))
            p = plan.poisson_solve(dev(f)).cpu().numpy()
            assert rel(p, ref) < tol, (case, d, rel(p, ref))
            if case % 4 == 0:  # the host-buffer entry point: the same bits
                ph = np.empty_like(f)
                plan.poisson_solve_host(np.ascontiguousarray(f), ph)
                assert np.array_equal(ph, p), case
            if not d["refined"]:  # stage by stage: the same bits as the solve
                x = dev(f)
                t = torch.empty_like(x)
                plan.poisson_stage(chanfs.X_FORWARD, x, out=t)
                for st in (chanfs.Y_FORWARD, chanfs.Z_SOLVE, chanfs.Y_INVERSE, chanfs.X_INVERSE):
                    plan.poisson_stage(st, t, out=t)
                assert np.array_equal(t.cpu().numpy(), p), case
            if d["ybc"] == 0 and case % 3 == 0:  # the fully implicit Helmholtz solve (Eq. 8)
                r3 = synth.normal(3000 + case, (nz, ny, nx))
                u3ref = oracle.helmholtz3d_solve(r3, lx, ly, dz, d["c"], d["loc"])
                u3 = plan.helmholtz3d_solve(d["c"], dev(r3), d["loc"]).cpu().numpy()
                assert rel(u3, u3ref) < tol, (case, d, rel(u3, u3ref))
            rhs = synth.normal(2000 + case, (nz, ny, nx))
            uref = oracle.helmholtz_solve(rhs, dz, d["c"], d["loc"])
            u = plan.helmholtz_solve(d["c"], dev(rhs), d["loc"]).cpu().numpy()
            assert rel(u, uref) < tol, (case, d, rel(u, uref))
            assert plan.check() == 0
            assert plan.check_guards() == 0
            ran += 1
    assert ran >= 72, (ran, skipped)


def test_random_groups_give_the_bits_of_solves_alone(chanfs):
    """Groups of 2 to 5 random refined plans (sizes, walls, kernel options,
    Helmholtz by FP64 Algorithm 2 or Thomas, refined in one pass or by the
    loop with FP32 Algorithm 2 or Thomas inner solves): every box's grouped
    Poisson and Helmholtz results equal its results alone, bit for bit,
    through direct launches, a graph capture and a replay."""
    rng = np.random.default_rng(602)
    groups = 0
    for g in range(12):
        plans, fs, rhs, alone_p, alone_u, cs, locs = [], [], [], [], [], [], []
        try:
            for b in range(int(rng.integers(2, 6))):
                d = draw(rng, chanfs)
                if not d["refined"]:
                    continue
                nx, ny, nz = d["nx"], d["ny"], d["nz"]
                dz = synth.uniform_dz(nz) if d["beta"] == 0.0 else synth.tanh_dz(nz, d["beta"])
                try:
                    pl = chanfs.Plan(nx, ny, nz, 2.0, 1.0, dz, d["bc"], chanfs.F32_REFINED,
                                     d["ybc"])
                except chanfs.ChanfsError as e:
                    assert e.status == chanfs.EUNSUPPORTED
                    continue
                plans.append(pl)
                for opt, key in ((chanfs.OPT_THOMAS_TILE, "thomas"),
                                 (chanfs.OPT_PCR_PARTS, "parts"),
                                 (chanfs.OPT_HELM_THOMAS, "helm_thomas"),
                                 (chanfs.OPT_HELM_FP64, "helm_fp64"),
                                 (chanfs.OPT_HELM_THOMAS32, "helm_thomas32")):
                    try:
                        pl.set_option(opt, d["opts"][key])
                    except chanfs.ChanfsError as e:
                        assert e.status == chanfs.EUNSUPPORTED
                f = synth.normal(3000 + 10 * g + b, (nz, ny, nx))
                if d["bc"] == 0 and d["ybc"] != 2:
                    f = synth.remove_weighted_mean(f, dz)
                fs.append(dev(f))
                rhs.append(dev(synth.normal(4000 + 10 * g + b, (nz, ny, nx))))
                cs.append(d["c"])
                locs.append(d["loc"])
                alone_p.append(pl.poisson_solve(fs[-1]).cpu().numpy())
                alone_u.append(pl.helmholtz_solve(cs[-1], rhs[-1], locs[-1]).cpu().numpy())
            if len(plans) < 2:
                continue
            with chanfs.Group(plans) as grp:
                for _ in range(3):
                    got_p = [o.cpu().numpy() for o in grp.poisson_solve(fs)]
                    got_u = [o.cpu().numpy() for o in grp.helmholtz_solve(cs, rhs, locs)]
                    for a, b in zip(got_p, alone_p):
                        assert np.array_equal(a, b), g
                    for a, b in zip(got_u, alone_u):
                        assert np.array_equal(a, b), g
            groups += 1
        finally:
            for pl in plans:
                pl.close()
    assert groups >= 4, groups


def test_random_slab_splits_match_the_oracle(chanfs):
    """z-slab solves (P-TDMA) of random grids split over 1 to 4 slabs on one
    GPU (the boundary buffers concatenated as the all-gather delivers them):
    Poisson and Helmholtz against the oracle at 1e-12."""
    rng = np.random.default_rng(2206)
    ran = 0
    for case in range(16):
        m = int(rng.choice([k for k in SMOOTH if 2 <= k <= 32]))
        nx, ny = 2 * m, int(rng.choice([k for k in SMOOTH if k <= 48]))
        R = int(rng.integers(1, 5))
        nz = int(rng.integers(6 * R, 90))
        bc = int(rng.integers(2))
        dz = synth.tanh_dz(nz, float(rng.uniform(1.0, 2.4)))
        lx, ly = 2.0, 1.5
        try:
            ss = [chanfs.Slab(nx, ny, nz, lx, ly, dz, bc, R, r) for r in range(R)]
        except chanfs.ChanfsError as e:
            assert e.status == chanfs.EUNSUPPORTED, (nx, ny, nz, R, e)
            continue
        try:
            f = synth.normal(5000 + case, (nz, ny, nx))
            if bc == 0:
                f = synth.remove_weighted_mean(f, dz)
            ref = oracle.poisson_solve(f, lx, ly, dz, bc)
            fl = [dev(f[s.z0:s.z1]) for s in ss]
            work = [torch.empty_like(x) for x in fl]
            bnd = [torch.empty(s.boundary_doubles(chanfs.REQ_POISSON), dtype=torch.float64,
                               device="cuda") for s in ss]
            for s, x, w, b in zip(ss, fl, work, bnd):
                s.poisson_reduce(x, w, b)
            outs = [torch.empty_like(x) for x in fl]
            for s, w, o in zip(ss, work, outs):
                s.poisson_finish(torch.cat(bnd), w, o)
            p = np.concatenate([o.cpu().numpy() for o in outs])
            assert rel(p, ref) < 1e-12, (case, nx, ny, nz, R, bc, rel(p, ref))
            c, loc = float(10.0 ** rng.uniform(-6, -2)), int(rng.integers(2))
            rhs = synth.normal(6000 + case, (nz, ny, nx))
            uref = oracle.helmholtz_solve(rhs, dz, c, loc)
            rl = [dev(rhs[s.z0:s.z1]) for s in ss]
            work = [torch.empty_like(x) for x in rl]
            bnd = [torch.empty(s.boundary_doubles(chanfs.REQ_HELMHOLTZ), dtype=torch.float64,
                               device="cuda") for s in ss]
            for s, x, w, b in zip(ss, rl, work, bnd):
                s.helmholtz_reduce(c, loc, x, w, b)
            outs = [torch.empty_like(x) for x in rl]
            for s, w, o in zip(ss, work, outs):
                s.helmholtz_finish(c, loc, torch.cat(bnd), w, o)
            u = np.concatenate([o.cpu().numpy() for o in outs])
            assert rel(u, uref) < 1e-12, (case, nx, ny, nz, R, loc, rel(u, uref))
            ran += 1
        finally:
            for s in ss:
                s.close()
    assert ran >= 12, ran
