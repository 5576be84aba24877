"""Helpers shared by the GPU parity tests (marshalling and error measures only)."""
import numpy as np


def rel_err(y, ref):
    """Norm-wise relative error ||y - ref||_inf / ||ref||_inf."""
    y = np.asarray(y, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(y - ref).max() / max(np.abs(ref).max(), 1e-300))


def to_np(t):
    import torch
    return t.detach().to(torch.float64).cpu().numpy()
