"""Failure paths of the solve entry points, made on the host side (no fault is
raised on the GPU): non-finite problem data comes back as KFBI_ERR_NONFINITE
from the single and the batched GMRES, a non-finite initial density is
dropped in favour of the zero start (x0_rejected), and the problem stays
usable after each failure."""
import numpy as np
import pytest

import workloads as W
from oracle import kfbi as OK
from tests.gpu_util import empty, gpu_data, host

pytestmark = pytest.mark.gpu

_cache = {}


def _flower():
    if "f" not in _cache:
        from paper_2309_05965_gb300 import build, kfbi
        build.build()
        w = W.flower_interface_2d(128)
        P = OK.Problem(w)
        G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED)
        data = W.grid_data(w)
        g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
        _cache["f"] = (w, P, G, data, g1, g2)
    return _cache["f"]


def _solve(G, d, x0=None, rtol=1e-10):
    from paper_2309_05965_gb300 import kfbi
    x = empty(G.nb)
    opts = kfbi.GmresOpts(rtol=rtol, restart=100, max_iter=100,
                          x0=None if x0 is None else x0.data_ptr())
    return kfbi.kfbi_gmres_solve(G.handle, d, opts, x), x


@pytest.mark.parametrize("where", ["g1", "g2", "f_in", "lapf_out"])
@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_nonfinite_data_is_reported(where, value):
    from paper_2309_05965_gb300 import kfbi
    w, P, G, data, g1, g2 = _flower()
    data = {k: v.copy() for k, v in data.items()}
    g1, g2 = g1.copy(), g2.copy()
    if where == "g1":
        g1[len(g1) // 3] = value
    elif where == "g2":
        g2[-1] = value
    else:
        # a node next to the interface, inside for f_in, outside for lapf_out
        sel = P.irr & (P.inside if where == "f_in" else ~P.inside)
        data[where][tuple(np.argwhere(sel)[0])] = value
    d, keep = gpu_data(w, P, data, g1, g2)
    with pytest.raises(kfbi.KfbiError) as e:
        _solve(G, d)
    assert e.value.status == 5, e.value
    # the problem is still usable: a clean solve afterwards converges
    d0, keep0 = gpu_data(w, P, _flower()[3], _flower()[4], _flower()[5])
    info, x = _solve(G, d0)
    assert info.rel_res <= 1e-10 and np.all(np.isfinite(host(x)))


def test_nonfinite_start_is_rejected():
    """A NaN in x0 makes ||b - A x0|| non-finite: the start is dropped and
    GMRES runs from zero, giving the zero-start result."""
    import torch
    w, P, G, data, g1, g2 = _flower()
    d, keep = gpu_data(w, P, data, g1, g2)
    info0, x_zero = _solve(G, d)
    x0 = torch.randn(G.nb, dtype=torch.float64, device="cuda")
    x0[5] = float("nan")
    info, x = _solve(G, d, x0)
    assert info.x0_rejected == 1
    assert info.iters == info0.iters
    assert np.array_equal(host(x), host(x_zero))


def test_nonfinite_batch_instance_is_reported():
    from paper_2309_05965_gb300 import kfbi
    w, P, G, data, g1, g2 = _flower()
    w2 = W.flower_interface_2d(256, contrast=10.0)
    P2 = OK.Problem(w2)
    G2 = kfbi.Problem.from_workload(w2, precision=kfbi.MIXED)
    data2 = W.grid_data(w2)
    a1, a2 = W.boundary_data(w2, P2.surf.x, P2.surf.n)
    a1 = a1.copy()
    a1[0] = np.nan
    d, keep = gpu_data(w, P, data, g1, g2)
    d2, keep2 = gpu_data(w2, P2, data2, a1, a2)
    B = kfbi.Batch([G, G2])
    opts = kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=100, x0=None)
    with pytest.raises(kfbi.KfbiError) as e:
        B.gmres_solve([d, d2], opts, [empty(G.nb), empty(G2.nb)])
    assert e.value.status == 5
    B.close()
    G2.close()
    info, x = _solve(G, d)
    assert info.rel_res <= 1e-10
