"""Helpers shared by the GPU parity tests."""
import numpy as np
import pytest
import torch

import paper_1602_02170_gb300 as mb


@pytest.fixture(scope="session")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = mb.Context(0)
    yield c
    c.close()


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype).contiguous()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
