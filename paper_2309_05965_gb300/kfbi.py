"""Thin Python binding of the C ABI in ``include/kfbi.h``.

Argument marshalling only: every computation runs in ``libkfbi.so`` on the GPU.
Device arrays are ``torch`` CUDA tensors (their ``data_ptr()`` is passed); the
CUDA stream is torch's current stream unless given.  There is no CPU path: if
the shared library has not been built or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkfbi.so")

KFBI_OK = 0
STATUS_NAMES = {0: "KFBI_OK", 1: "KFBI_ERR_ARG", 2: "KFBI_ERR_GEOMETRY", 3: "KFBI_ERR_SINGULAR",
                4: "KFBI_ERR_NOT_CONVERGED", 5: "KFBI_ERR_NONFINITE", 6: "KFBI_ERR_TIMEOUT",
                7: "KFBI_ERR_CUDA", 8: "KFBI_ERR_UNSUPPORTED"}
LS_MAX_PARAMS = 64

DIRICHLET_INTERIOR = 0
INTERFACE_MU = 1
NEUMANN_INTERIOR = 2
INTERFACE_GENERAL = 3
BOX_DST = 0
BOX_MG = 1
FP64 = 0
MIXED = 1


class KfbiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class LevelSet(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_params", ctypes.c_int),
                ("p", ctypes.c_double * LS_MAX_PARAMS), ("samples", ctypes.c_void_p)]


class Config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("lo", ctypes.c_double),
                ("hi", ctypes.c_double), ("order", ctypes.c_int), ("kind", ctypes.c_int),
                ("sigma_in", ctypes.c_double), ("sigma_out", ctypes.c_double),
                ("kappa", ctypes.c_double), ("box_solver", ctypes.c_int),
                ("precision", ctypes.c_int), ("cos_alpha", ctypes.c_double),
                ("box_rtol", ctypes.c_double), ("box_max_iters", ctypes.c_int),
                ("kappa_out", ctypes.c_double), ("relax", ctypes.c_double)]


class Data(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("g1", "g2", "f_in", "f_out", "lapf_in", "lapf_out", "g_b")] + \
        [("in_per_interface", ctypes.c_int)]


class GmresOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("x0", ctypes.c_void_p)]


class GmresInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("t_ms", ctypes.c_double * 8), ("x0_rejected", ctypes.c_int),
                ("refine_steps", ctypes.c_int)]


# name -> (argtypes) ; all return kfbi_status except kfbi_last_error
_P = ctypes.c_void_p
_I = ctypes.POINTER(ctypes.c_int)
SIGNATURES = {
    "kfbi_create_problem": [ctypes.POINTER(Config), ctypes.POINTER(LevelSet), _P,
                            ctypes.POINTER(ctypes.c_void_p)],
    "kfbi_destroy_problem": [_P],
    "kfbi_update_levelset": [_P, ctypes.POINTER(LevelSet)],
    "kfbi_sizes": [_P, _I, _I, _I],
    "kfbi_num_dofs": [_P, _I],
    "kfbi_dof_points": [_P, _P, _P],
    "kfbi_dof_info": [_P, _P, _P, _P],
    "kfbi_stencil_sizes": [_P, _I, _I, _I],
    "kfbi_collocation_stencils": [_P, _P, _P, _P],
    "kfbi_inside_mask": [_P, _P],
    "kfbi_irregular_nodes": [_P, _P, _P],
    "kfbi_interfaces": [_P, _I, _I],
    "kfbi_dof_iface": [_P, _P],
    "kfbi_correction_entries": [_P, _P, _P, _P],
    "kfbi_collocation_fit": [_P, _P, _P, _P, _P],
    "kfbi_correction_values": [_P, _P, _P, _P, _P],
    "kfbi_corrected_rhs": [_P, _P, ctypes.POINTER(Data), _P],
    "kfbi_box_solve": [_P, _P, _P],
    "kfbi_traces": [_P, _P, _P, _P, _P, _P, _P],
    "kfbi_apply_operator": [_P, _P, _P],
    "kfbi_bie_rhs": [_P, ctypes.POINTER(Data), _P],
    "kfbi_gmres_solve": [_P, ctypes.POINTER(Data), ctypes.POINTER(GmresOpts), _P,
                         ctypes.POINTER(GmresInfo)],
    "kfbi_evaluate": [_P, ctypes.POINTER(Data), _P, _P],
    "kfbi_create_batch": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)],
    "kfbi_destroy_batch": [_P],
    "kfbi_batch_tiles": [_P, _I, _I],
    "kfbi_gmres_solve_batch": [_P, _P, ctypes.POINTER(GmresOpts), _P, _P, _P],
    "kfbi_evaluate_batch": [_P, _P, _P, _P],
    "kfbi_mlp_create": [ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_void_p)],
    "kfbi_mlp_destroy": [_P],
    "kfbi_mlp_num_params": [_P, _I],
    "kfbi_mlp_set_params": [_P, _P],
    "kfbi_mlp_get_params": [_P, _P, _P],
    "kfbi_mlp_set_affine": [_P, _P, _P, ctypes.c_double, ctypes.c_double],
    "kfbi_mlp_forward": [_P, _P, ctypes.c_int, _P],
    "kfbi_mlp_loss_grad": [_P, _P, _P, _P, ctypes.c_int, _P],
    "kfbi_mlp_adam": [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float],
    "kfbi_mlp_set_trainable": [_P, ctypes.c_int],
    "kfbi_warm_start_features": [_P, ctypes.POINTER(Data), _P, _P, _P],
    "kfbi_warm_start": [_P, _P, ctypes.POINTER(Data), _P],
    "kfbi_warm_start_batch": [_P, _P, _P, _P],
    "kfbi_box_solve_noalloc": [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_int, ctypes.c_double, _P, _P, _P],
    "kfbi_box_solve_info": [_P, _P, _P, _P, _P],
    "kfbi_launch_counts": [_P, _P, ctypes.c_int],
    "kfbi_profile_enable": [_P, ctypes.c_int],
    "kfbi_profile_read": [_P, _P, _P],
}

KERNEL_CLASSES = ["correction", "rhs", "dst", "residual", "mg", "trace", "gmres", "other"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libkfbi.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: the CUDA library must be built "
                           "(paper_2309_05965_gb300.build.build()) — there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.kfbi_last_error.argtypes = [_P]
    lib.kfbi_last_error.restype = ctypes.c_char_p
    lib.kfbi_mlp_last_error.argtypes = [_P]
    lib.kfbi_mlp_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device arrays must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("device arrays must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check(status: int, handle=None):
    if status != KFBI_OK:
        msg = load().kfbi_last_error(handle)
        raise KfbiError(status, msg.decode() if msg else "")


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---- the C entry points under their own names ------------------------------

def kfbi_create_problem(cfg: Config, ls: LevelSet, stream=None):
    h = ctypes.c_void_p()
    _check(load().kfbi_create_problem(ctypes.byref(cfg), ctypes.byref(ls),
                                      _stream_handle(stream), ctypes.byref(h)))
    return h


def kfbi_destroy_problem(h):
    _check(load().kfbi_destroy_problem(h))


def kfbi_sizes(h):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().kfbi_sizes(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), h)
    return a.value, b.value, c.value


def kfbi_stencil_sizes(h):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().kfbi_stencil_sizes(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), h)
    return a.value, b.value, c.value


def kfbi_dof_points(h, xyz, normals):
    _check(load().kfbi_dof_points(h, _ptr(xyz), _ptr(normals)), h)


def kfbi_dof_info(h, family, axis, stencil_axis):
    _check(load().kfbi_dof_info(h, _ptr(family), _ptr(axis), _ptr(stencil_axis)), h)


def kfbi_collocation_stencils(h, pde, dirs, neus):
    _check(load().kfbi_collocation_stencils(h, _ptr(pde), _ptr(dirs), _ptr(neus)), h)


def kfbi_inside_mask(h, mask):
    _check(load().kfbi_inside_mask(h, _ptr(mask)), h)


def kfbi_irregular_nodes(h, lin, owner):
    _check(load().kfbi_irregular_nodes(h, _ptr(lin), _ptr(owner)), h)


def kfbi_interfaces(h):
    n_iface, n_ent = ctypes.c_int(), ctypes.c_int()
    _check(load().kfbi_interfaces(h, ctypes.byref(n_iface), ctypes.byref(n_ent)), h)
    return n_iface.value, n_ent.value


def kfbi_dof_iface(h, iface):
    _check(load().kfbi_dof_iface(h, _ptr(iface)), h)


def kfbi_correction_entries(h, lin, iface, owner):
    _check(load().kfbi_correction_entries(h, _ptr(lin), _ptr(iface), _ptr(owner)), h)


def kfbi_collocation_fit(h, a, b, ftilde, coef):
    _check(load().kfbi_collocation_fit(h, _ptr(a), _ptr(b), _ptr(ftilde), _ptr(coef)), h)


def kfbi_correction_values(h, a, b, ftilde, cvals):
    _check(load().kfbi_correction_values(h, _ptr(a), _ptr(b), _ptr(ftilde), _ptr(cvals)), h)


def make_data(g1=None, g2=None, f_in=None, f_out=None, lapf_in=None, lapf_out=None, g_b=None,
              in_per_interface=False):
    """kfbi_data from device tensors; in_per_interface: f_in and lapf_in hold
    one grid per interface (a leading axis of length n_iface)."""
    d = Data()
    for k, v in (("g1", g1), ("g2", g2), ("f_in", f_in), ("f_out", f_out),
                 ("lapf_in", lapf_in), ("lapf_out", lapf_out), ("g_b", g_b)):
        p = _ptr(v)
        setattr(d, k, p.value if p is not None else None)
    d.in_per_interface = int(bool(in_per_interface))
    return d


def kfbi_corrected_rhs(h, cvals, data, rhs):
    _check(load().kfbi_corrected_rhs(h, _ptr(cvals), ctypes.byref(data) if data else None,
                                     _ptr(rhs)), h)


def kfbi_box_solve(h, rhs, u):
    _check(load().kfbi_box_solve(h, _ptr(rhs), _ptr(u)), h)


def kfbi_traces(h, u, cvals, vp=None, vm=None, dp=None, dm=None):
    _check(load().kfbi_traces(h, _ptr(u), _ptr(cvals), _ptr(vp), _ptr(vm), _ptr(dp), _ptr(dm)), h)


def kfbi_apply_operator(h, x, y):
    _check(load().kfbi_apply_operator(h, _ptr(x), _ptr(y)), h)


def kfbi_bie_rhs(h, data, b):
    _check(load().kfbi_bie_rhs(h, ctypes.byref(data), _ptr(b)), h)


def kfbi_gmres_solve(h, data, opts: GmresOpts, density):
    info = GmresInfo()
    _check(load().kfbi_gmres_solve(h, ctypes.byref(data), ctypes.byref(opts), _ptr(density),
                                   ctypes.byref(info)), h)
    return info


def kfbi_evaluate(h, data, density, u):
    _check(load().kfbi_evaluate(h, ctypes.byref(data), _ptr(density), _ptr(u)), h)


def kfbi_create_batch(handles):
    """Batch over problem handles (errors are reported on handles[0])."""
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    b = ctypes.c_void_p()
    _check(load().kfbi_create_batch(ctypes.cast(arr, ctypes.c_void_p), len(handles),
                                    ctypes.byref(b)), handles[0])
    return b


def kfbi_destroy_batch(b):
    _check(load().kfbi_destroy_batch(b))


def kfbi_batch_tiles(b):
    """(pass_ctas, row_ctas): the launch shapes chosen when the batch was created."""
    pc, rc = ctypes.c_int(), ctypes.c_int()
    _check(load().kfbi_batch_tiles(b, ctypes.byref(pc), ctypes.byref(rc)))
    return pc.value, rc.value


def kfbi_gmres_solve_batch(b, handles, datas, opts: GmresOpts, densities, x0s=None):
    """Algorithm 1 for every instance (x0s: None, or one tensor or None per
    instance); returns one GmresInfo per instance."""
    n = len(handles)
    darr = (Data * n)(*datas)
    parr = (ctypes.c_void_p * n)(*[_ptr(x).value for x in densities])
    xarr = None
    if x0s is not None:
        xarr = (ctypes.c_void_p * n)(*[(_ptr(x).value if x is not None else None) for x in x0s])
    infos = (GmresInfo * n)()
    _check(load().kfbi_gmres_solve_batch(b, ctypes.cast(darr, ctypes.c_void_p), ctypes.byref(opts),
                                         ctypes.cast(xarr, ctypes.c_void_p) if xarr is not None else None,
                                         ctypes.cast(parr, ctypes.c_void_p),
                                         ctypes.cast(infos, ctypes.c_void_p)), handles[0])
    return list(infos)


def kfbi_evaluate_batch(b, handles, datas, densities, u_grids):
    """Grid solution of every instance from its density (one batched box solve)."""
    n = len(handles)
    darr = (Data * n)(*datas)
    parr = (ctypes.c_void_p * n)(*[_ptr(x).value for x in densities])
    uarr = (ctypes.c_void_p * n)(*[_ptr(x).value for x in u_grids])
    _check(load().kfbi_evaluate_batch(b, ctypes.cast(darr, ctypes.c_void_p), ctypes.cast(parr, ctypes.c_void_p),
                                      ctypes.cast(uarr, ctypes.c_void_p)), handles[0])


WS_FEATURES = 16   # KFBI_WS_FEATURES


def _check_mlp(status, m):
    if status != KFBI_OK:
        msg = load().kfbi_mlp_last_error(m)
        raise KfbiError(status, msg.decode() if msg else "")


def kfbi_mlp_create(n_in, width, stream=None):
    m = ctypes.c_void_p()
    _check(load().kfbi_mlp_create(n_in, width, _stream_handle(stream), ctypes.byref(m)))
    return m


def kfbi_mlp_destroy(m):
    _check(load().kfbi_mlp_destroy(m))


def kfbi_mlp_num_params(m):
    c = ctypes.c_int()
    _check_mlp(load().kfbi_mlp_num_params(m, ctypes.byref(c)), m)
    return c.value


def kfbi_mlp_set_params(m, params):
    _check_mlp(load().kfbi_mlp_set_params(m, _ptr(params)), m)


def kfbi_mlp_get_params(m, params=None, grads=None):
    _check_mlp(load().kfbi_mlp_get_params(m, _ptr(params), _ptr(grads)), m)


def kfbi_mlp_set_affine(m, in_shift, in_scale, out_shift, out_scale):
    import numpy as np
    a = np.ascontiguousarray(in_shift, dtype=np.float32)
    b = np.ascontiguousarray(in_scale, dtype=np.float32)
    _check_mlp(load().kfbi_mlp_set_affine(m, a.ctypes.data_as(ctypes.c_void_p),
                                          b.ctypes.data_as(ctypes.c_void_p), float(out_shift),
                                          float(out_scale)), m)


def kfbi_mlp_forward(m, X, y):
    _check_mlp(load().kfbi_mlp_forward(m, _ptr(X), int(X.shape[0]), _ptr(y)), m)


def kfbi_mlp_loss_grad(m, X, t, rows=None, loss=None, n=None):
    """Gradient over the rows `rows` (int32 device tensor) of X, t, or all rows."""
    count = int(rows.shape[0]) if rows is not None else int(X.shape[0] if n is None else n)
    _check_mlp(load().kfbi_mlp_loss_grad(m, _ptr(X), _ptr(t), _ptr(rows), count, _ptr(loss)), m)


MLP_BRANCH, MLP_LINEAR = 1, 2


def kfbi_mlp_set_trainable(m, groups):
    _check_mlp(load().kfbi_mlp_set_trainable(m, groups), m)


def kfbi_mlp_adam(m, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check_mlp(load().kfbi_mlp_adam(m, lr, beta1, beta2, eps), m)


def kfbi_warm_start_features(h, data, features, density=None, target=None):
    _check(load().kfbi_warm_start_features(h, ctypes.byref(data), _ptr(density), _ptr(features),
                                           _ptr(target)), h)


def kfbi_warm_start(h, m, data, x0):
    _check(load().kfbi_warm_start(h, m, ctypes.byref(data), _ptr(x0)), h)


def kfbi_box_solve_info(h):
    """(steps, cycles, rel_change, converged) of the last box solve on h."""
    st, cy, cv = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rel = ctypes.c_double()
    _check(load().kfbi_box_solve_info(h, ctypes.byref(st), ctypes.byref(cy), ctypes.byref(rel),
                                      ctypes.byref(cv)), h)
    return st.value, cy.value, rel.value, cv.value


def kfbi_box_solve_noalloc(dim, n, lo, hi, order, kappa, rhs, u, stream=None):
    """FP64 DST box solve with no device allocation (fixed library scratch)."""
    _check(load().kfbi_box_solve_noalloc(dim, n, lo, hi, order, kappa, _ptr(rhs), _ptr(u),
                                         _stream_handle(stream)))


def kfbi_launch_counts(h, reset=False):
    arr = (ctypes.c_int64 * len(KERNEL_CLASSES))()
    _check(load().kfbi_launch_counts(h, ctypes.cast(arr, ctypes.c_void_p), int(reset)), h)
    return dict(zip(KERNEL_CLASSES, list(arr)))


def kfbi_profile_enable(h, on=True):
    _check(load().kfbi_profile_enable(h, int(on)), h)


def kfbi_profile_read(h):
    ms = (ctypes.c_double * len(KERNEL_CLASSES))()
    cnt = (ctypes.c_int64 * len(KERNEL_CLASSES))()
    _check(load().kfbi_profile_read(h, ctypes.cast(ms, ctypes.c_void_p),
                                    ctypes.cast(cnt, ctypes.c_void_p)), h)
    return {k: (m, c) for k, m, c in zip(KERNEL_CLASSES, list(ms), list(cnt))}


# ---- convenience object ------------------------------------------------------

class Problem:
    """Owns one kfbi_problem.  Sizes and shapes are read back at creation."""

    def __init__(self, dim, n, lo, hi, ls_kind, ls_params, kind, sigma_in=1.0, sigma_out=1.0,
                 kappa=0.0, order=4, box_solver=BOX_DST, precision=FP64, cos_alpha=0.0,
                 box_rtol=0.0, box_max_iters=0, stream=None, kappa_out=0.0, ls_samples=None,
                 relax=0.0):
        cfg = Config(dim=dim, n=n, lo=lo, hi=hi, order=order, kind=kind, sigma_in=sigma_in,
                     sigma_out=sigma_out, kappa=kappa, box_solver=box_solver,
                     precision=precision, cos_alpha=cos_alpha, box_rtol=box_rtol,
                     box_max_iters=box_max_iters, kappa_out=kappa_out, relax=relax)
        ls = LevelSet(kind=ls_kind, n_params=len(ls_params))
        for i, v in enumerate(ls_params):
            ls.p[i] = float(v)
        keep = None
        if ls_samples is not None:
            # node values of a grid-sampled level set: a device copy for the
            # call (the library copies them at create)
            import numpy as np
            import torch
            keep = (ls_samples if isinstance(ls_samples, torch.Tensor) else
                    torch.as_tensor(np.ascontiguousarray(ls_samples, dtype=np.float64)).cuda())
            ls.samples = keep.data_ptr()
        self.cfg = cfg
        self.dim, self.n = dim, n
        self.handle = kfbi_create_problem(cfg, ls, stream)
        del keep
        self.nb, self.nirr, self.ncoef = kfbi_sizes(self.handle)
        self.n_iface, self.nent = kfbi_interfaces(self.handle)
        self.npde, self.ndir, self.nneu = kfbi_stencil_sizes(self.handle)

    def update_levelset(self, ls_kind, ls_params, ls_samples=None):
        """A new interface on the same grid (kfbi_update_levelset); sizes are
        read back."""
        ls = LevelSet(kind=ls_kind, n_params=len(ls_params))
        for i, v in enumerate(ls_params):
            ls.p[i] = float(v)
        keep = None
        if ls_samples is not None:
            import numpy as np
            import torch
            keep = (ls_samples if isinstance(ls_samples, torch.Tensor) else
                    torch.as_tensor(np.ascontiguousarray(ls_samples, dtype=np.float64)).cuda())
            ls.samples = keep.data_ptr()
        _check(load().kfbi_update_levelset(self.handle, ctypes.byref(ls)), self.handle)
        del keep
        self.nb, self.nirr, self.ncoef = kfbi_sizes(self.handle)
        self.n_iface, self.nent = kfbi_interfaces(self.handle)

    @classmethod
    def from_workload(cls, w, box_solver=BOX_DST, precision=FP64, **kw):
        return cls(w.dim, w.n, w.lo, w.hi, w.ls_kind, w.ls_params, w.kind,
                   sigma_in=w.sigma_in, sigma_out=w.sigma_out, kappa=w.kappa, order=w.order,
                   box_solver=box_solver, precision=precision,
                   cos_alpha=w.cos_alpha or 0.0, kappa_out=w.kappa_out,
                   ls_samples=w.extra.get("samples"), **kw)

    def close(self):
        if self.handle is not None:
            kfbi_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def grid_shape(self):
        return (self.n + 1,) * self.dim


class Batch:
    """Owns one kfbi_batch over Problem objects (kept alive by the batch)."""

    def __init__(self, problems):
        self.problems = list(problems)
        self.handle = kfbi_create_batch([q.handle for q in self.problems])

    def gmres_solve(self, datas, opts: GmresOpts, densities, x0s=None):
        return kfbi_gmres_solve_batch(self.handle, [q.handle for q in self.problems], datas, opts,
                                      densities, x0s)

    def evaluate(self, datas, densities, u_grids):
        kfbi_evaluate_batch(self.handle, [q.handle for q in self.problems], datas, densities, u_grids)

    def warm_start(self, mlp, datas, x0s):
        """Every instance's start from one forward pass of the network."""
        n = len(self.problems)
        darr = (Data * n)(*datas)
        xarr = (ctypes.c_void_p * n)(*[_ptr(x).value for x in x0s])
        _check(load().kfbi_warm_start_batch(self.handle, mlp, ctypes.cast(darr, ctypes.c_void_p),
                                            ctypes.cast(xarr, ctypes.c_void_p)), self.problems[0].handle)

    def tiles(self):
        return kfbi_batch_tiles(self.handle)

    def close(self):
        if self.handle is not None:
            kfbi_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
