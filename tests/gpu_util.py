"""Helpers shared by the GPU parity tests: host <-> device marshalling of the
column-major FP64 arrays the C ABI takes, and the error measures."""
import numpy as np

U64 = np.finfo(np.float64).eps / 2


def dev(a):
    """numpy (any order) -> column-major FP64 CUDA tensor."""
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    if a.size == 0:
        return torch.zeros(a.shape, dtype=torch.float64, device="cuda")
    t = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()   # (cols, rows) row-major
    return t.t()                                             # (rows, cols), stride (1, rows)


def host(t):
    return t.detach().cpu().numpy().copy() if t.dim() == 1 else t.detach().cpu().numpy().copy(order="F")


def zeros(n):
    import torch
    return torch.zeros(n, dtype=torch.float64, device="cuda")


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb else 1.0)
