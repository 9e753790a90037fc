"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the
FP64 oracle on identical seeded inputs)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def have_gpu():
    return torch.cuda.is_available()


def dev():
    return torch.device("cuda:0")


def t32(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev())


def to_np(t):
    return t.detach().double().cpu().numpy()


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def csr_t(rp, ci, va, dtype=None):
    return (torch.tensor(rp, dtype=torch.int64, device=dev()),
            torch.tensor(ci, dtype=torch.int32, device=dev()),
            torch.tensor(va, dtype=dtype or torch.float32, device=dev()))
