"""Helpers shared by the GPU parity tests: run the oracle and the CUDA library
on the same seeded workload and move arrays between them."""
import numpy as np

import workloads as W


def torch_mod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def dev(a, dtype=None):
    torch = torch_mod()
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch_mod().cuda.synchronize()
    return t.detach().cpu().numpy()


def empty(shape, dtype="f64"):
    torch = torch_mod()
    dt = {"f64": torch.float64, "i32": torch.int32, "u8": torch.uint8, "f32": torch.float32}[dtype]
    return torch.zeros(shape, dtype=dt, device="cuda")


def rel_err(a, b):
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / scale)


def linear_nodes(idx, n):
    """multi-index (..., d) -> linear C-order index of the (N+1)^d grid."""
    idx = np.asarray(idx)
    lin = idx[..., 0].astype(np.int64)
    for k in range(1, idx.shape[-1]):
        lin = lin * (n + 1) + idx[..., k]
    return lin


def gpu_data(w, P_or, data, g1, g2):
    """Device copies of the problem data and a kfbi_data struct."""
    from paper_2309_05965_gb300 import kfbi
    keep = {}
    for k in ("f_in", "f_out", "lapf_in", "lapf_out", "g_b"):
        keep[k] = dev(data[k])
    keep["g1"] = dev(g1) if g1 is not None else None
    keep["g2"] = dev(g2) if g2 is not None else None
    d = kfbi.make_data(g1=keep["g1"], g2=keep["g2"], f_in=keep["f_in"], f_out=keep["f_out"],
                       lapf_in=keep["lapf_in"], lapf_out=keep["lapf_out"],
                       g_b=keep["g_b"] if w.kind in (W.KIND_INTERFACE_MU, W.KIND_INTERFACE_GENERAL) else None,
                       in_per_interface=data["f_in"].ndim == w.dim + 1)
    return d, keep
