"""The manufactured data of the workloads against finite differences of their
closed forms: f = sigma Lap u - kappa u on each side and Lap f, for every
exact solution the workloads use.  Both the oracle and the CUDA path take
these inputs, so parity could not catch a wrong closed form; this can."""
import numpy as np
import pytest

import workloads as W


def _lap(F, h, d):
    """Second-order 3/5/7-point Laplacian on the interior nodes."""
    inner = tuple(slice(1, -1) for _ in range(d))
    L = -2.0 * d * F[inner]
    for ax in range(d):
        lo = [slice(1, -1)] * d
        hi = [slice(1, -1)] * d
        lo[ax] = slice(0, -2)
        hi[ax] = slice(2, None)
        L = L + F[tuple(lo)] + F[tuple(hi)]
    return L / (h * h)


CASES = [
    lambda: W.ellipse_dirichlet_2d(64),
    lambda: W.paper_table1_2d(64),
    lambda: W.flower_interface_2d(64),
    lambda: W.torus_helmholtz_3d(32),
    lambda: W.neumann_torus_3d(32),
    lambda: W.neumann_torus_3d(32, kappa=2.0),
    lambda: W.neumann_ellipse_2d(64, 1.0),
    lambda: W.hetero_interface_2d(64),
    lambda: W.hetero_sphere_3d(32),
    lambda: W.discs_interface_2d(64),
]


@pytest.mark.parametrize("make", CASES)
def test_sources_match_finite_differences(make):
    w = make()
    d, h = w.dim, w.h
    g = W.grid_data(w)
    X = W.grid_coords(w)
    (ui, _, _), (uo, _, _) = W.solutions(w)
    inner = tuple(slice(1, -1) for _ in range(d))
    sides = [("in", ui, w.sigma_in, w.kappa)]
    if w.kind in (W.KIND_INTERFACE_MU, W.KIND_INTERFACE_GENERAL):
        k_out = w.kappa_out if w.kind == W.KIND_INTERFACE_GENERAL else 0.0
        sides.append(("out", uo, w.sigma_out, k_out))
    for name, u, sigma, kappa in sides:
        U = u(X)
        f_fd = sigma * _lap(U, h, d) - kappa * U[inner]
        f = g["f_" + name][inner]
        scale = max(1.0, float(np.abs(f).max()))
        assert np.abs(f_fd - f).max() < 2e-2 * scale, (w.name, name)
        lf_fd = _lap(g["f_" + name], h, d)
        lf = g["lapf_" + name][inner]
        scale = max(1.0, float(np.abs(lf).max()))
        assert np.abs(lf_fd - lf).max() < 5e-2 * scale, (w.name, name)


@pytest.mark.parametrize("make", [lambda: W.neumann_ellipse_2d(64), lambda: W.hetero_interface_2d(64)])
def test_flux_data_match_finite_differences(make):
    """g_N = sigma d_n u (Neumann) and g2 = [sigma d_n u] (interfaces) from
    the closed-form gradients against central differences along the normal."""
    w = make()
    t = np.linspace(0.0, 2.0 * np.pi, 17)[:-1]
    pts = np.stack([0.3 * np.cos(t), 0.2 * np.sin(t)], -1)
    nrm = np.stack([np.cos(t), np.sin(t)], -1)
    (ui, _, _), (uo, _, _) = W.solutions(w)
    e = 1e-5
    dn_i = (ui(pts + e * nrm) - ui(pts - e * nrm)) / (2 * e)
    dn_o = (uo(pts + e * nrm) - uo(pts - e * nrm)) / (2 * e)
    g1, g2 = W.boundary_data(w, pts, nrm)
    if w.kind == W.KIND_NEUMANN:
        ref = w.sigma_in * dn_i
    else:
        ref = w.sigma_in * dn_i - w.sigma_out * dn_o
        assert np.abs(g1 - (ui(pts) - uo(pts))).max() < 1e-14
    assert np.abs(g2 - ref).max() < 1e-8


def test_wave_fields_are_harmonic_with_exact_gradients():
    import numpy as np
    import workloads as W
    w = W.wave_ellipsoid_3d([0.5, 0.4, 0.6], 64)
    (ui, gi, li), (uo, go, lo) = W.solutions(w)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, size=(40, 3))
    e = 1e-4
    for u, g in ((ui, gi), (uo, go)):
        lap = -6 * u(X)
        for k in range(3):
            d = np.zeros(3)
            d[k] = e
            assert np.abs((u(X + d) - u(X - d)) / (2 * e) - g(X)[:, k]).max() < 1e-6
            lap = lap + u(X + d) + u(X - d)
        assert np.abs(lap / (e * e)).max() < 1e-4
    assert np.abs(ui(X) - uo(X)).max() > 0.1
