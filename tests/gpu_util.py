"""Helpers for the GPU parity tests: numpy <-> CUDA tensors in the library's
layout (row k of an (nrhs, n) array is right-hand side k)."""
import numpy as np


def to_dev(a):
    import torch
    a = np.ascontiguousarray(np.atleast_2d(a), dtype=np.complex128)
    return torch.from_numpy(a).to("cuda")


def to_host(t):
    return t.cpu().numpy()


def empty(nrhs, n):
    import torch
    return torch.empty((nrhs, n), dtype=torch.complex128, device="cuda")


def zeros(nrhs, n):
    import torch
    return torch.zeros((nrhs, n), dtype=torch.complex128, device="cuda")


def col_rel(got, want):
    """Relative 2-norm error per right-hand side (rows of (nrhs, n) arrays)."""
    got = np.atleast_2d(got)
    want = np.atleast_2d(want)
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
