"""Helpers for the GPU parity tests (inputs from synthdata, references from oracle)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ctx(**params):
    import paper_2401_06747_b300 as hdi
    return hdi.Context(0, **params)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()
