"""Helpers for the GPU tests: device tensors from Python ints (uint64 bit
patterns stored in int64 tensors)."""
import numpy as np


def u64_tensor(values, device="cuda:0"):
    import torch
    a = np.array([int(v) & ((1 << 64) - 1) for v in values], dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64)).to(device)


def u32_tensor(values, device="cuda:0"):
    import torch
    a = np.array([int(v) for v in values], dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).to(device)


def to_u64_list(t):
    return [int(x) for x in t.cpu().numpy().view(np.uint64)]


def to_u32_list(t):
    return [int(x) for x in t.cpu().numpy().view(np.uint32)]
