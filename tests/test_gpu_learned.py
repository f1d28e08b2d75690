"""The learned initial density: network kernels against the oracle network
(forward, loss, gradient, Adam), and the gain of the trained network over the
zero start of GMRES on held-out problems."""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as OM
from tests.gpu_util import empty, host

pytestmark = pytest.mark.gpu


def _net(width=256, seed=7):
    import torch
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    rng = np.random.default_rng(seed)
    ni = kfbi.WS_FEATURES
    P = OM.Params(rng.standard_normal((width, ni)) * 0.4, rng.standard_normal(width) * 0.1,
                  rng.standard_normal((width, width)) / np.sqrt(width),
                  rng.standard_normal(width) * 0.1, rng.standard_normal((1, width)) / np.sqrt(width),
                  rng.standard_normal(1) * 0.1, rng.standard_normal((1, ni)) * 0.3)
    flat32 = P.flat().astype(np.float32)
    P = OM.Params.from_flat(flat32.astype(np.float64), ni, width)
    m = kfbi.kfbi_mlp_create(ni, width)
    assert kfbi.kfbi_mlp_num_params(m) == flat32.size
    kfbi.kfbi_mlp_set_params(m, torch.from_numpy(flat32).cuda())
    kfbi.kfbi_mlp_set_affine(m, np.zeros(ni), np.ones(ni), 0.0, 1.0)
    return m, P, rng


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("n", [1, 63, 1000])
def test_forward_loss_and_gradient_match_oracle(n):
    """FP32 sums of bf16-rounded weights against the FP64 oracle with the same
    rounded weights: outputs and gradients to FP32 accumulation accuracy over
    ragged row counts (one row, under one tile, several tiles)."""
    import torch
    from paper_2309_05965_gb300 import kfbi
    m, P, rng = _net()
    X = rng.standard_normal((n, kfbi.WS_FEATURES)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    y = empty(n, "f32")
    kfbi.kfbi_mlp_forward(m, Xd, y)
    y_ref, _ = OM.forward(P, X.astype(np.float64))
    assert _rel(host(y), y_ref) < 2e-5
    loss = empty(1, "f32")
    kfbi.kfbi_mlp_loss_grad(m, Xd, td, loss=loss)
    L_ref, G_ref = OM.loss_and_grad(P, X.astype(np.float64), t.astype(np.float64))
    assert abs(float(host(loss)[0]) - L_ref) <= 2e-5 * L_ref
    g = empty(kfbi.kfbi_mlp_num_params(m), "f32")
    kfbi.kfbi_mlp_get_params(m, grads=g)
    gg = OM.Params.from_flat(host(g).astype(np.float64), kfbi.WS_FEATURES, 256)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "WL"):
        assert _rel(getattr(gg, name), getattr(G_ref, name)) < 1e-4, name
    kfbi.kfbi_mlp_destroy(m)


def test_minibatch_rows_and_adam_step_match_oracle():
    """A gathered minibatch gives the oracle's gradient on those rows, and one
    Adam step moves the parameters as the oracle's Adam does."""
    import torch
    from paper_2309_05965_gb300 import kfbi
    m, P, rng = _net(seed=11)
    n = 700
    X = rng.standard_normal((n, kfbi.WS_FEATURES)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    rows = rng.permutation(n)[:257].astype(np.int32)
    kfbi.kfbi_mlp_loss_grad(m, torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(),
                            rows=torch.from_numpy(rows).cuda())
    _, G_ref = OM.loss_and_grad(P, X[rows].astype(np.float64), t[rows].astype(np.float64))
    npar = kfbi.kfbi_mlp_num_params(m)
    g = empty(npar, "f32")
    th0 = empty(npar, "f32")
    kfbi.kfbi_mlp_get_params(m, params=th0, grads=g)
    assert _rel(host(g), G_ref.flat()) < 1e-4
    lr = 1e-3
    kfbi.kfbi_mlp_adam(m, lr, 0.9, 0.999, 1e-8)
    th1 = empty(npar, "f32")
    kfbi.kfbi_mlp_get_params(m, params=th1)
    gh = host(g).astype(np.float64)
    ref, _, _ = OM.adam_step(host(th0).astype(np.float64), gh, np.zeros(npar), np.zeros(npar), 1, lr)
    step = host(th1).astype(np.float64) - host(th0).astype(np.float64)
    want = ref - host(th0).astype(np.float64)
    # FP32 parameters: the step is resolved to the FP32 spacing of the parameter
    tol = 1e-3 * lr + 2.0 * np.spacing(np.abs(host(th0)).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(step - want) <= tol)
    kfbi.kfbi_mlp_destroy(m)


def _family_solve(kfbi, G, w, opts, x, x0=None):
    """Boundary data of the harmonic family at the DOFs, then one solve."""
    import torch
    xyz = torch.zeros((G.nb, 3), dtype=torch.float64, device="cuda")
    nrm = torch.zeros((G.nb, 3), dtype=torch.float64, device="cuda")
    kfbi.kfbi_dof_points(G.handle, xyz, nrm)
    g1, g2 = W.boundary_data(w, xyz.cpu().numpy(), nrm.cpu().numpy())
    grid = W.grid_data(w)
    keep = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in
            (("g1", g1), ("g2", g2), ("f_in", grid["f_in"]), ("f_out", grid["f_out"]),
             ("lapf_in", grid["lapf_in"]), ("lapf_out", grid["lapf_out"]), ("g_b", grid["g_b"]))}
    d = kfbi.make_data(**keep)
    o = kfbi.GmresOpts(rtol=opts.rtol, restart=opts.restart, max_iter=opts.max_iter,
                       x0=None if x0 is None else x0.data_ptr())
    info = kfbi.kfbi_gmres_solve(G.handle, d, o, x)
    return info, d, keep


def test_trained_warm_start_beats_zero_start():
    """Train on the library's solves of the wave-field ellipsoid family (64^3,
    60 ellipsoids drawn, unresolved ones skipped: fixed non-polynomial
    harmonic fields inside and outside, so the density is neither an input
    feature nor a multiple of one), then on held-out ellipsoids: the learned
    start is taken, needs fewer GMRES iterations, reaches the same solution
    and keeps the error against the exact solution; a useless start is
    rejected in favour of zero."""
    import torch
    from paper_2309_05965_gb300 import build, kfbi, learned
    build.build()
    n = 64
    opts = kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=100, x0=None)
    ds = learned.Dataset(60 * 12000)
    for axes in W.ellipsoid_axes(101, 60):
        w = W.wave_ellipsoid_3d(axes, n)
        try:
            G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED)
        except kfbi.KfbiError as e:
            assert e.status == 2   # an ellipsoid the grid cannot resolve
            continue
        x = empty(G.nb)
        _, d, keep = _family_solve(kfbi, G, w, opts, x)
        ds.add(G, d, x)
        G.close()
    assert ds.solves >= 40
    ws = learned.WarmStart(seed=3)
    hist = ws.fit(ds, epochs=16, batch=2048, lr=2e-3, lr_final=1e-6, min_steps=6000)
    assert ws.branch_trained, "the density is not linear in the features: the branch must train"
    assert hist[-1] < 0.05 * hist[0]
    gains = []
    held = [a for a in W.ellipsoid_axes(202, 12) if min(a) > 0.4][:3]
    for axes in held:
        w = W.wave_ellipsoid_3d(axes, n)
        G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED)
        x_zero = empty(G.nb)
        info0, d, keep = _family_solve(kfbi, G, w, opts, x_zero)
        x0 = empty(G.nb)
        ws.predict(G, d, x0)
        # the start is a real approximation of the solved density
        assert float((x0 - x_zero).abs().max() / x_zero.abs().max()) < 0.05
        x_l = empty(G.nb)
        info1, _, _ = _family_solve(kfbi, G, w, opts, x_l, x0=x0)
        assert info1.x0_rejected == 0
        gains.append(info0.iters - info1.iters)
        assert float((x_l - x_zero).abs().max() / x_zero.abs().max()) < 1e-8
        # the error against the exact solution is the zero start's
        ins = torch.zeros(G.grid_shape, dtype=torch.uint8, device="cuda")
        kfbi.kfbi_inside_mask(G.handle, ins)
        ex = W.exact_grid(w, host(ins).astype(bool))
        u0, u1 = empty(G.grid_shape), empty(G.grid_shape)
        kfbi.kfbi_evaluate(G.handle, d, x_zero, u0)
        kfbi.kfbi_evaluate(G.handle, d, x_l, u1)
        e0 = np.abs(host(u0) - ex)[1:-1, 1:-1, 1:-1].max()
        e1 = np.abs(host(u1) - ex)[1:-1, 1:-1, 1:-1].max()
        assert e1 <= 1.1 * e0, (e1, e0)
        # a useless start (huge) is dropped: same iterations as zero start
        bad = torch.full_like(x0, 1e6)
        x_b = empty(G.nb)
        info2, _, _ = _family_solve(kfbi, G, w, opts, x_b, x0=bad)
        assert info2.x0_rejected == 1 and info2.iters == info0.iters
        G.close()
    assert min(gains) >= 2, gains
    ws.close()


def test_learned_starts_in_a_batch():
    """The learned + mixed + batched form on star interfaces (the batched
    configuration's family, reading of its data: u_in = sin x cos y, u_out =
    x^2 + y^2, contrast 10^U[0,3]): a network trained on 40 problems of one
    seed gives the starts of a batch of other problems; every start is taken,
    every instance needs fewer iterations than from zero, and the solutions
    agree with the zero-start batch and keep its error."""
    import torch
    from paper_2309_05965_gb300 import build, kfbi, learned
    build.build()
    opts = kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=100, x0=None)

    def instances(seed, count):
        out = []
        for w in W.star_batch_2d(count=4 * count, seed=seed, sizes=(128, 256)):
            if len(out) == count:
                break
            try:
                G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED)
            except kfbi.KfbiError as e:
                assert e.status == 2
                continue
            out.append((w, G))
        return out

    def data(w, G):
        xyz, nrm = empty((G.nb, 2)), empty((G.nb, 2))
        kfbi.kfbi_dof_points(G.handle, xyz, nrm)
        g1, g2 = W.boundary_data(w, host(xyz), host(nrm))
        grid = W.grid_data(w)
        keep = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in
                (("g1", g1), ("g2", g2), ("f_in", grid["f_in"]), ("f_out", grid["f_out"]),
                 ("lapf_in", grid["lapf_in"]), ("lapf_out", grid["lapf_out"]), ("g_b", grid["g_b"]))}
        return kfbi.make_data(**keep), keep

    train = instances(11, 40)
    ds = learned.Dataset(sum(G.nb for _, G in train))
    for w, G in train:
        d, keep = data(w, G)
        x = empty(G.nb)
        kfbi.kfbi_gmres_solve(G.handle, d, opts, x)
        ds.add(G, d, x)
        G.close()
    ws = learned.WarmStart(seed=4)
    hist = ws.fit(ds, epochs=16, batch=4096, lr=2e-3, lr_final=1e-6, min_steps=6000)
    assert ws.branch_trained and hist[-1] < 0.05 * hist[0]
    rows = instances(12, 6)
    dd = [data(w, G) for w, G in rows]
    B = kfbi.Batch([G for _, G in rows])
    xz = [empty(G.nb) for _, G in rows]
    iz = B.gmres_solve([d for d, _ in dd], opts, xz)
    x0s = [empty(G.nb) for _, G in rows]
    for (w, G), (d, _), x0 in zip(rows, dd, x0s):
        ws.predict(G, d, x0)
    # one forward pass over every instance's DOFs gives the same starts
    xb = [empty(G.nb) for _, G in rows]
    ws.predict_batch(B, [d for d, _ in dd], xb)
    for a, b in zip(x0s, xb):
        assert float((a - b).abs().max()) <= 1e-6 * float(a.abs().max())
    xl = [empty(G.nb) for _, G in rows]
    il = B.gmres_solve([d for d, _ in dd], opts, xl, x0s=x0s)
    uz = [empty(G.grid_shape) for _, G in rows]
    ul = [empty(G.grid_shape) for _, G in rows]
    B.evaluate([d for d, _ in dd], xz, uz)
    B.evaluate([d for d, _ in dd], xl, ul)
    for k, ((w, G), a, b) in enumerate(zip(rows, iz, il)):
        assert b.x0_rejected == 0 and b.iters < a.iters, (k, a.iters, b.iters)
        assert float((xl[k] - xz[k]).abs().max() / xz[k].abs().max()) < 1e-6
        ins = torch.zeros(G.grid_shape, dtype=torch.uint8, device="cuda")
        kfbi.kfbi_inside_mask(G.handle, ins)
        ex = W.exact_grid(w, host(ins).astype(bool))
        e0 = np.abs(host(uz[k]) - ex)[1:-1, 1:-1].max()
        e1 = np.abs(host(ul[k]) - ex)[1:-1, 1:-1].max()
        assert e1 <= 1.1 * e0 + 1e-12, (k, e1, e0)
    B.close()
    for _, G in rows:
        G.close()
    ws.close()
