"""The box solve that allocates nothing, for callers that may not call
cudaMalloc themselves (their device memory belongs to a host application or
pool, or an allocation there could stall or fail mid-pipeline).

Called through the C ABI (kfbi_box_solve_noalloc) and checked against the
regular entry point kfbi_box_solve of a problem on the same grid, within the
FP64 box-solve tolerance of the parity suite, on two calls in a row (the
shared scratch keeps the previous call's contents), and against the oracle's
sine-transform solve.  The largest accepted grids (2D N = 512, 3D N = 64,
whose work grid fills the fixed scratch exactly) are included, and one call
runs on a side stream.  This file is collected last so that a run stopping at
its first failure has run everything else.
"""
import numpy as np
import pytest

import workloads as W
from oracle import boxsolve as BS

pytestmark = pytest.mark.gpu


def _kappa(w):
    return w.kappa / w.sigma_in if w.kind == W.KIND_DIRICHLET else w.kappa


def _regular(w, R):
    from paper_2309_05965_gb300 import kfbi
    from tests.gpu_util import dev, empty, host
    G = kfbi.Problem.from_workload(w, box_solver=kfbi.BOX_DST, precision=kfbi.FP64)
    u = empty(G.grid_shape)
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    out = host(u)
    G.close()
    return out


def _noalloc(w, R, stream=None):
    from paper_2309_05965_gb300 import kfbi
    from tests.gpu_util import dev, empty, host
    u = empty((w.n + 1,) * w.dim)
    kfbi.kfbi_box_solve_noalloc(w.dim, w.n, w.lo, w.hi, w.order, _kappa(w), dev(R), u, stream)
    if stream is not None:
        stream.synchronize()
    return host(u)


def _ell3(n):
    return W.Workload("ell3", 3, n, -1.0, 1.0, W.LS_ELLIPSOID, [0.05, -0.03, 0.02, 0.8, 0.7, 0.6],
                      W.KIND_DIRICHLET, kappa=1.0, exact="exp3")


def test_noalloc_matches_box_solve_on_consecutive_calls():
    from paper_2309_05965_gb300 import build
    from tests.gpu_util import rel_err
    build.build()
    w2 = W.ellipse_dirichlet_2d(256)
    w2.kappa = 3.0
    w3 = _ell3(32)
    cases = [(w2, W.sine_grid_rhs(2, 256, 11)), (w3, W.sine_grid_rhs(3, 32, 12)),
             (w2, W.sine_grid_rhs(2, 256, 13))]
    for w, R in cases:
        a = _noalloc(w, R)
        b = _regular(w, R)
        assert rel_err(a, b) < 1e-12


def test_noalloc_largest_sizes_against_oracle():
    """2D N = 512 and 3D N = 64 (the largest accepted), two calls in a row,
    each against kfbi_box_solve and against the oracle's DST-I solve; the
    second 3D call on a side stream."""
    import torch
    from paper_2309_05965_gb300 import build
    from tests.gpu_util import rel_err
    build.build()
    w2 = W.ellipse_dirichlet_2d(512)
    w2.kappa = 2.0
    w3 = _ell3(64)
    w3o2 = _ell3(64)
    w3o2.order = 2
    side = torch.cuda.Stream()
    cases = [(w2, W.sine_grid_rhs(2, 512, 21), None), (w3, W.sine_grid_rhs(3, 64, 22), None),
             (w3o2, W.sine_grid_rhs(3, 64, 23), side)]
    for w, R, st in cases:
        a = _noalloc(w, R, st)
        b = _regular(w, R)
        ref = BS.dst_solve(R, w.dim, w.order, w.h, _kappa(w))
        assert rel_err(a, b) < 1e-12
        assert rel_err(a, ref) < 1e-12
        for ax in range(w.dim):
            assert np.all(np.take(a, [0, w.n], axis=ax) == 0.0)


def test_noalloc_rejects_sizes_beyond_its_scratch_and_aliasing():
    from paper_2309_05965_gb300 import build, kfbi
    from tests.gpu_util import empty
    build.build()
    big = empty((1025, 1025))
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.kfbi_box_solve_noalloc(2, 1024, -1.0, 1.0, 4, 0.0, big, big)
    assert e.value.status == 1
    cube = empty((129, 129, 129))
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.kfbi_box_solve_noalloc(3, 128, -1.0, 1.0, 4, 0.0, cube, cube)
    assert e.value.status == 1
    # rhs and u overlapping (the same grid, or shifted by one node): refused
    # before any work is enqueued, the input left as it was
    g = empty((2 * 65 * 65,))
    g[: 65 * 65] = 1.0
    for off in (0, 1):
        with pytest.raises(kfbi.KfbiError) as e:
            kfbi.kfbi_box_solve_noalloc(2, 64, -1.0, 1.0, 4, 0.0, g[: 65 * 65], g[off: off + 65 * 65])
        assert e.value.status == 1
    assert float(g[: 65 * 65].min()) == 1.0
