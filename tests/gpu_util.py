"""Helpers shared by the GPU tests: host <-> device transfers and the
normwise relative error used for parity."""
import numpy as np


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().to("cpu").double().numpy()


def rel_err(x, ref):
    """||x - ref||_inf / ||ref||_inf."""
    x, ref = np.asarray(x, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    den = np.abs(ref).max()
    return float(np.abs(x - ref).max() / (den if den > 0 else 1.0))


def faces_or_none(u):
    return None if u is None else dev(u)
