"""GPU: every output element of every entry point is written.

Outputs start as NaN (a poisoned buffer); after each call no NaN may remain,
and the result must equal that of a second call into a zeroed buffer (so an
element the kernels skip, or one they read before writing, shows up).  Sizes
mix radix-3 lengths, a single y cell, z columns shorter than the in-thread
prefetch, and tiles with a ragged tail.
"""

import numpy as np
import pytest

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


SIZES = [(6, 9, 5), (24, 27, 7), (48, 1, 4), (12, 6, 33), (96, 18, 3)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def written(fn, like):
    """fn(out) into a NaN-poisoned and into a zeroed buffer: both equal, no NaN."""
    poisoned = torch.full_like(like, float("nan"))
    fn(poisoned)
    clean = torch.zeros_like(like)
    fn(clean)
    torch.cuda.synchronize()
    a, b = poisoned.cpu().numpy(), clean.cpu().numpy()
    assert not np.isnan(a).any(), f"{np.isnan(a).sum()} elements left unwritten"
    assert np.array_equal(a, b)
    return a


@pytest.mark.parametrize("dims", SIZES)
@pytest.mark.parametrize("dtype", [0, 1])
def test_every_element_is_written(chanfs, dims, dtype):
    nx, ny, nz = dims
    if dtype == 1 and nx % 4:
        pytest.skip("refined plans need nx % 4 == 0")
    dz = synth.tanh_dz(nz, 1.4)
    f = dev(synth.remove_weighted_mean(synth.normal(3 * nx + nz, (nz, ny, nx)), dz))
    with chanfs.Plan(nx, ny, nz, 2.0, 1.5, dz, chanfs.NEUMANN, dtype) as plan:
        written(lambda o: plan.poisson_solve(f, out=o), f)
        thomas_opt = chanfs.OPT_HELM_THOMAS32 if dtype == 1 else chanfs.OPT_HELM_THOMAS
        for method in (0, 1):
            plan.set_option(thomas_opt, method)
            for loc in (chanfs.CENTER, chanfs.FACE):
                if nz - loc < 3:
                    continue  # Algorithm 2 needs 3 rows per partition
                u = written(lambda o: plan.helmholtz_solve(1e-3, f, loc, out=o), f)
                if loc == chanfs.FACE:
                    assert np.all(u[-1] == 0.0)
        for loc in (chanfs.CENTER, chanfs.FACE):
            written(lambda o: plan.helmholtz3d_solve(2e-3, f, loc, out=o), f)
        if dtype == 0:
            s = written(lambda o: plan.spectral_forward(f, out=o), f)
            written(lambda o: plan.spectral_inverse(dev(s), out=o), f)
        assert plan.check() == 0


@pytest.mark.parametrize("ybc", [1, 2])
def test_every_element_is_written_with_y_walls(chanfs, ybc):
    for nx, ny, nz in SIZES[:3]:
        dz = synth.tanh_dz(nz, 1.4)
        f = dev(synth.normal(5 * ny + nz, (nz, ny, nx)))
        with chanfs.Plan(nx, ny, nz, 2.0, 1.5, dz, chanfs.DIRICHLET, chanfs.F64, ybc) as plan:
            written(lambda o: plan.poisson_solve(f, out=o), f)
            written(lambda o: plan.helmholtz3d_solve(1e-3, f, chanfs.CENTER, out=o), f)
            assert plan.check() == 0


def test_every_element_is_written_by_grouped_solves(chanfs):
    specs = [(24, 27, 7), (12, 6, 33), (96, 18, 5), (48, 1, 4)]
    plans, fs = [], []
    for i, (nx, ny, nz) in enumerate(specs):
        dz = synth.tanh_dz(nz, 1.3 + 0.2 * i)
        plans.append(chanfs.Plan(nx, ny, nz, 2.0, 1.5, dz, chanfs.NEUMANN, chanfs.F32_REFINED))
        fs.append(dev(synth.remove_weighted_mean(synth.normal(40 + i, (nz, ny, nx)), dz)))
    plans[1].set_option(chanfs.OPT_HELM_THOMAS32, 1)
    plans[2].set_option(chanfs.OPT_HELM_FP64, 1)
    with chanfs.Group(plans) as g:
        for _ in range(2):  # direct launches, then a graph
            outs = [torch.full_like(x, float("nan")) for x in fs]
            g.poisson_solve(fs, outs)
            for o in outs:
                assert not torch.isnan(o).any()
            outs = [torch.full_like(x, float("nan")) for x in fs]
            g.helmholtz_solve([1e-3] * 4, fs, [chanfs.FACE] * 4, outs)
            for o in outs:
                assert not torch.isnan(o).any()
                assert torch.all(o[-1] == 0)
    for p in plans:
        p.close()
