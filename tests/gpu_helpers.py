"""Helpers for the GPU tests: move numpy arrays through the C ABI with torch
device buffers.  Only the tests import this module."""
import numpy as np


def torch_dev():
    import torch

    return torch, torch.device("cuda:0")


def stream():
    torch, dev = torch_dev()
    return torch.cuda.current_stream(dev).cuda_stream


def to_dev_real(a: np.ndarray):
    torch, dev = torch_dev()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)


def to_dev_c64(a: np.ndarray):
    """complex array -> device float32 tensor with a trailing (re, im) axis."""
    torch, dev = torch_dev()
    a = np.ascontiguousarray(a, dtype=np.complex64)
    return torch.from_numpy(a.view(np.float32).reshape(a.shape + (2,))).to(dev)


def from_dev_c64(t) -> np.ndarray:
    a = t.detach().cpu().numpy()
    return np.ascontiguousarray(a).view(np.complex64)[..., 0]


def empty_c64(shape):
    torch, dev = torch_dev()
    return torch.empty(tuple(shape) + (2,), dtype=torch.float32, device=dev)


def empty_real(shape):
    torch, dev = torch_dev()
    return torch.empty(tuple(shape), dtype=torch.float32, device=dev)


def sync():
    torch, dev = torch_dev()
    torch.cuda.synchronize(dev)


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
