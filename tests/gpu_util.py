"""Helpers shared by the GPU parity tests."""
import numpy as np


def rel_fro(a, b) -> float:
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def gpu_apply(h, X):
    """H_eff X through the device entry point (X: (nvec, dim) host array)."""
    import torch
    X = np.atleast_2d(X)
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    yd = torch.full_like(xd, float("nan"))
    h.apply(xd, yd, nvec=X.shape[0])
    torch.cuda.synchronize()
    return yd.cpu().numpy()
