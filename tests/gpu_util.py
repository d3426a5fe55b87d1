"""Helpers shared by the GPU parity tests (marshalling only)."""
import numpy as np
import torch


def to_dev(a, device="cuda"):
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint64:
        a = a.astype(np.int64).view(np.uint64)
    return torch.from_numpy(a.view(np.int64).copy()).to(device)


def to_np(t):
    return t.detach().cpu().contiguous().numpy().view(np.uint64)


def as_u64(obj_arr):
    return np.array(obj_arr, dtype=object).astype(np.uint64)
