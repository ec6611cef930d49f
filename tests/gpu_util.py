"""Helpers for the GPU tests (marshalling only: no arithmetic of the method)."""
import numpy as np


def to_dev(F):
    import torch
    return torch.as_tensor(np.ascontiguousarray(F), device="cuda")


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()
