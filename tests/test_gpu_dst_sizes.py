"""Box solve by sine transform at every transform length the kernels
instantiate (L = 2N from 16 to 4096): FP64 path and mixed path (FP32
transforms, FP64 residuals, refinement) against the oracle's DST-I solve on a
seeded random right-hand side, and against the closed form on single sine
modes (eigenvectors of the compact operators: u = R / lambda, lambda the
stencil's symbol sum_o c_o prod_k cos(p_k pi o_k / N))."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import boxsolve as BS
from tests.gpu_util import dev, empty, host, rel_err

pytestmark = pytest.mark.gpu

# (dim, N, order): every LOGL = log2(2N) from 4 to 12, 2D and 3D
SIZES = [(2, 8, 2), (2, 16, 2), (3, 16, 2), (2, 32, 4), (3, 32, 4), (2, 64, 4), (3, 64, 4),
         (2, 128, 4), (3, 128, 4), (2, 256, 4), (3, 256, 4), (2, 512, 4), (2, 1024, 4),
         (2, 2048, 4)]
ORACLE_MAX = {2: 1024, 3: 256}   # sizes where the oracle's full solve is compared


def _problem(d, n, order, precision):
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    if d == 2:
        w = W.Workload("box", 2, n, -1.0, 1.0, W.LS_ELLIPSE, [0.0, 0.0, 0.7, 0.6, 0.0],
                       W.KIND_DIRICHLET, kappa=1.0, exact="exp_sin")
    else:
        w = W.Workload("box", 3, n, -1.0, 1.0, W.LS_ELLIPSOID, [0.0, 0.0, 0.0, 0.75, 0.7, 0.65],
                       W.KIND_DIRICHLET, kappa=1.0, exact="exp3")
    w.order = order
    G = kfbi.Problem.from_workload(w, precision=precision, box_max_iters=8)
    return w, G


def _mixed_tol(n):
    # FP32 transforms contract the error by about eps32 * cond(A_h) per step,
    # cond ~ 4 N^2 / pi^2, eight steps at most; the FP64 residual itself
    # resolves u only to ~eps64 * cond(A_h)
    c = 6e-8 * 0.45 * n * n
    return max(5e-12, 1e-17 * n * n, 10.0 * c ** 8)


def _symbol(d, order, n, h, kappa, modes):
    c = BS.stencil_coeffs(d, order, h, kappa)
    lam = 0.0
    for o in itertools.product((-1, 0, 1), repeat=d):
        w = c[sum(1 for v in o if v != 0)]
        lam += w * np.prod([np.cos(p * np.pi * ok / n) for p, ok in zip(modes, o)])
    return lam


@pytest.mark.parametrize("d,n,order", SIZES)
@pytest.mark.parametrize("precision", [0, 1])
def test_dst_random_rhs_matches_oracle(d, n, order, precision):
    if n > ORACLE_MAX[d]:
        pytest.skip("full oracle solve only up to the listed sizes")
    from paper_2309_05965_gb300 import kfbi
    w, G = _problem(d, n, order, precision)
    R = W.sine_grid_rhs(d, n, 17)
    ref = BS.dst_solve(R, d, order, w.h, w.kappa)
    u = empty(G.grid_shape)
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    tol = 1e-12 if precision == 0 else _mixed_tol(n)
    assert rel_err(host(u), ref) < tol
    G.close()


@pytest.mark.parametrize("d,n,order", SIZES)
@pytest.mark.parametrize("precision", [0, 1])
def test_dst_sine_modes_closed_form(d, n, order, precision):
    import torch
    from paper_2309_05965_gb300 import kfbi
    w, G = _problem(d, n, order, precision)
    for modes in ([1] * d, [n - 1] * d, [n // 2 + 1, 3, n - 2][:d], [2, n - 1, n // 3][:d]):
        R = torch.ones(G.grid_shape, dtype=torch.float64, device="cuda")
        for k, p in enumerate(modes):
            shape = [1] * d
            shape[k] = n + 1
            # reduce p i modulo 2N exactly first: an FP64 argument p pi i / N
            # of size ~p pi carries an absolute error ~1e-13 that is not an
            # eigenvector and that A_h^{-1} amplifies by cond(A_h)
            arg = torch.remainder(p * torch.arange(n + 1, device="cuda"), 2 * n).double()
            R = R * torch.sin(np.pi * arg / n).reshape(shape)
        lam = _symbol(d, order, n, w.h, w.kappa, modes)
        u = empty(G.grid_shape)
        kfbi.kfbi_box_solve(G.handle, R.contiguous(), u)
        want = R / lam
        # the symbol itself carries cancellation ~ eps64 * cond for low modes
        cond = 0.45 * n * n
        tol = (1e-12 if precision == 0 else _mixed_tol(n)) + 4e-16 * cond
        err = float((u - want).abs().max() / want.abs().max())
        assert err < tol, (modes, err)
    G.close()


@pytest.mark.parametrize("d,n,order", [(2, 256, 4), (3, 64, 4)])
def test_mixed_output_paths(d, n, order):
    """Where the mixed box solve writes its FP64 output: with no correction
    step (the conversion kernel), after a refinement that stops early on the
    convergence flag (the next residual kernel), and for a zero right-hand
    side (flag set after the first solve: u = 0 exactly, boundary included)."""
    import torch
    from paper_2309_05965_gb300 import kfbi
    R = W.sine_grid_rhs(d, n, 5)
    w, G1 = _problem(d, n, order, 1)
    G1.close()
    ref = BS.dst_solve(R, d, order, w.h, w.kappa)
    # one FP32 solve, no refinement: FP32-level accuracy
    G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED, box_max_iters=1)
    u = empty(G.grid_shape).fill_(7.0)
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    e1 = rel_err(host(u), ref)
    # one FP32 solve: error ~ eps32 cond(A_h) (cond ~ 0.45 N^2), not refined
    assert 1e-12 < e1 < 10 * 6e-8 * 0.45 * n * n, e1
    for ax in range(d):
        assert np.all(np.take(host(u), [0, n], axis=ax) == 0.0)
    G.close()
    # up to 8 steps at tol 1e-13: stops early, the output comes from u_fix
    G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED, box_max_iters=8)
    u = empty(G.grid_shape).fill_(7.0)
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    assert rel_err(host(u), ref) < _mixed_tol(n)
    for ax in range(d):
        assert np.all(np.take(host(u), [0, n], axis=ax) == 0.0)
    # zero right-hand side on the same problem: exactly zero
    u.fill_(7.0)
    kfbi.kfbi_box_solve(G.handle, torch.zeros(G.grid_shape, dtype=torch.float64, device="cuda"), u)
    assert float(u.abs().max()) == 0.0
    # and a normal solve afterwards is unaffected by the converged state
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    assert rel_err(host(u), ref) < _mixed_tol(n)
    G.close()


def test_largest_2d_grid():
    """N = 4096 in 2D (transform length 8192, the largest the library takes):
    the FP64 passes' shared memory does not fit a CTA, so FP64 is refused at
    create; the mixed path (one padded FP32 buffer per line pair) runs.  At
    this size eps32 cond(A_h) ~ 0.45, so its refinement converges slowly for
    high modes; low modes, whose FP32 solve is accurate, are reproduced in
    closed form."""
    import torch
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    n = 4096
    w = W.Workload("box", 2, n, -1.0, 1.0, W.LS_ELLIPSE, [0.0, 0.0, 0.7, 0.6, 0.0],
                   W.KIND_DIRICHLET, kappa=1.0, exact="exp_sin")
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.Problem.from_workload(w, precision=kfbi.FP64)
    assert e.value.status == 8
    G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED, box_max_iters=8)
    for modes in ([1, 1], [3, 2], [5, 1]):
        R = torch.ones(G.grid_shape, dtype=torch.float64, device="cuda")
        for k, p in enumerate(modes):
            shape = [1, 1]
            shape[k] = n + 1
            arg = torch.remainder(p * torch.arange(n + 1, device="cuda"), 2 * n).double()
            R = R * torch.sin(np.pi * arg / n).reshape(shape)
        lam = _symbol(2, 4, n, w.h, w.kappa, modes)
        u = empty(G.grid_shape)
        kfbi.kfbi_box_solve(G.handle, R.contiguous(), u)
        err = float((u - R / lam).abs().max() / (R / lam).abs().max())
        assert err < 1e-9, (modes, err)
    # a high mode: bounded and finite (slow refinement, see above)
    R = torch.ones(G.grid_shape, dtype=torch.float64, device="cuda")
    for k, p in enumerate([n - 1, n // 2 + 1]):
        shape = [1, 1]
        shape[k] = n + 1
        arg = torch.remainder(p * torch.arange(n + 1, device="cuda"), 2 * n).double()
        R = R * torch.sin(np.pi * arg / n).reshape(shape)
    lam = _symbol(2, 4, n, w.h, w.kappa, [n - 1, n // 2 + 1])
    u = empty(G.grid_shape)
    kfbi.kfbi_box_solve(G.handle, R.contiguous(), u)
    assert bool(torch.isfinite(u).all())
    assert float((u - R / lam).abs().max() / (R / lam).abs().max()) < 0.1
    G.close()


def test_box_solve_info_counts_the_work_that_ran():
    """kfbi_box_solve_info: the FP64 transform is one step; the mixed
    transform runs its first FP32 solve plus refinement steps until the flag
    stops it (fewer than the limit at tolerance 1e-13 for a smooth grid, all of
    them when the limit is small), one step for a zero right-hand side; the
    multigrid reports inner_cycles = 4 V-cycles per outer step (mixed) and the
    V-cycles it ran (FP64)."""
    import torch
    from paper_2309_05965_gb300 import kfbi
    n = 256
    R = W.sine_grid_rhs(2, n, 5)
    w, G = _problem(2, n, 4, 0)
    u = empty(G.grid_shape)
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    assert kfbi.kfbi_box_solve_info(G.handle)[:2] == (1, 0)
    G.close()
    for limit in (2, 8):
        G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED, box_max_iters=limit)
        kfbi.kfbi_box_solve(G.handle, dev(R), u)
        steps, cycles, rel, conv = kfbi.kfbi_box_solve_info(G.handle)
        assert cycles == 0 and 1 <= steps <= limit
        if limit == 2:
            assert steps == 2
        else:
            assert conv == 1 and steps < limit and rel <= 1e-13
        kfbi.kfbi_box_solve(G.handle, torch.zeros_like(u), u)
        assert kfbi.kfbi_box_solve_info(G.handle)[0] == 1
        G.close()
    for prec in (kfbi.FP64, kfbi.MIXED):
        G = kfbi.Problem.from_workload(w, box_solver=kfbi.BOX_MG, precision=prec)
        kfbi.kfbi_box_solve(G.handle, dev(R), u)
        steps, cycles, rel, conv = kfbi.kfbi_box_solve_info(G.handle)
        assert conv == 1 and cycles >= 2
        if prec == kfbi.MIXED:
            assert cycles == 4 * steps
        else:
            assert steps == 1
        G.close()
