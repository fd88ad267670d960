"""Helpers for the GPU tests: device tensors and parameter blocks.  No method
arithmetic lives here."""
import numpy as np


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    return torch


def dev(a, dtype):
    torch = torch_cuda()
    t = torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")
    return t.contiguous()


def empty(shape, dtype):
    torch = torch_cuda()
    return torch.empty(shape, dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().double().numpy()


def rel_fro(a, b):
    """Relative Frobenius error of two tensors given as 6-vectors
    [k11, k22, k33, k12, k23, k13] (off-diagonals counted twice)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    w = np.array([1, 1, 1, 2, 2, 2], dtype=np.float64)
    return float(np.sqrt((w * (a - b) ** 2).sum() / (w * b ** 2).sum()))
