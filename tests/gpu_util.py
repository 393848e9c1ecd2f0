"""Helpers shared by the GPU tests: a GPU gate and the oracle comparison."""
import numpy as np
import pytest

import oracle


def require_gpu():
    try:
        import torch
        ok = torch.cuda.is_available()
    except Exception:
        ok = False
    if not ok:
        pytest.skip("no CUDA device")


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_params(shape, h, dt, w, g, mode):
    return oracle.Params.make(shape, h, dt, w[0], w[1], w[2], g, mode)
