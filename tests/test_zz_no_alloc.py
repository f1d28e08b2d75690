"""The box solve that allocates nothing, for callers that may not call
cudaMalloc themselves (their device memory belongs to a host application or
pool, or an allocation there could stall or fail mid-pipeline).

Called through the C ABI (kfbi_box_solve_noalloc) and checked against the
regular entry point kfbi_box_solve of a problem on the same grid, within the
FP64 box-solve tolerance of the parity suite, on two calls in a row (the
shared scratch keeps the previous call's contents).  This file is collected
last so that a run stopping at its first failure has run everything else.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _regular(w, R):
    from paper_2309_05965_gb300 import kfbi
    from tests.gpu_util import dev, empty, host
    G = kfbi.Problem.from_workload(w, box_solver=kfbi.BOX_DST, precision=kfbi.FP64)
    u = empty(G.grid_shape)
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    out = host(u)
    G.close()
    return out


def _noalloc(w, R):
    from paper_2309_05965_gb300 import kfbi
    from tests.gpu_util import dev, empty, host
    kt = w.kappa / w.sigma_in if w.kind == W.KIND_DIRICHLET else w.kappa
    u = empty((w.n + 1,) * w.dim)
    kfbi.kfbi_box_solve_noalloc(w.dim, w.n, w.lo, w.hi, w.order, kt, dev(R), u)
    return host(u)


def test_noalloc_matches_box_solve_on_consecutive_calls():
    from paper_2309_05965_gb300 import build
    from tests.gpu_util import rel_err
    build.build()
    w2 = W.ellipse_dirichlet_2d(256)
    w2.kappa = 3.0
    w3 = W.Workload("ell3", 3, 32, -1.0, 1.0, W.LS_ELLIPSOID, [0.05, -0.03, 0.02, 0.8, 0.7, 0.6],
                    W.KIND_DIRICHLET, kappa=1.0, exact="exp3")
    cases = [(w2, W.sine_grid_rhs(2, 256, 11)), (w3, W.sine_grid_rhs(3, 32, 12)),
             (w2, W.sine_grid_rhs(2, 256, 13))]
    for w, R in cases:
        a = _noalloc(w, R)
        b = _regular(w, R)
        assert rel_err(a, b) < 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
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
