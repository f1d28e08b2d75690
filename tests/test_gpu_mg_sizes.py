"""3D multigrid box solve against the oracle's DST-I solve of the same
compact operator, at grids whose interior (N - 1 = 31, 63, 127 nodes per
axis) leaves ragged tiles in every 3D kernel (32-column, 16-row tiles of the
smoothing sweeps; per-level z-chunks), FP64 V-cycles and FP32 V-cycles inside
the exact fixed-point refinement, 27-point (4th order) and 7-point (2nd
order) operators.  The multigrid converges to the discrete solution, so the
comparison is element by element at the inner tolerance."""
import numpy as np
import pytest

import workloads as W
from oracle import boxsolve as BS
from tests.gpu_util import dev, empty, host, rel_err

pytestmark = pytest.mark.gpu


def _problem(n, order, precision):
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    w = W.Workload("box3", 3, n, -1.0, 1.0, W.LS_ELLIPSOID, [0.0, 0.0, 0.0, 0.75, 0.7, 0.65],
                   W.KIND_DIRICHLET, kappa=1.0, exact="exp3")
    w.order = order
    G = kfbi.Problem.from_workload(w, box_solver=kfbi.BOX_MG, precision=precision)
    return w, G


@pytest.mark.parametrize("n,order", [(32, 4), (64, 4), (128, 4), (64, 2)])
@pytest.mark.parametrize("precision", [0, 1])
def test_mg_box_solve_matches_dst_oracle(n, order, precision):
    from paper_2309_05965_gb300 import kfbi
    w, G = _problem(n, order, precision)
    R = W.sine_grid_rhs(3, n, 17)
    ref = BS.dst_solve(R, 3, order, w.h, w.kappa)
    u = empty(G.grid_shape)
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    got = host(u)
    assert rel_err(got, ref) < 1e-11, rel_err(got, ref)
    # boundary layer untouched (homogeneous Dirichlet)
    for ax in range(3):
        assert np.all(np.take(got, [0, n], axis=ax) == 0.0)
    # a second solve on the same problem gives the same result (state reset)
    u2 = empty(G.grid_shape)
    kfbi.kfbi_box_solve(G.handle, dev(R), u2)
    assert np.array_equal(host(u2), got)
    G.close()
