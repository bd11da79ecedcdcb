"""Helpers shared by the GPU tests: build the library once, share seeded inputs."""
import numpy as np
import pytest

from paper_1703_04789_gb300 import inputs


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


_built = {}


def library():
    if "lib" not in _built:
        from paper_1703_04789_gb300 import build
        _built["lib"] = build.build()
    return _built["lib"]


def masked_random_two_site(ql, qr, rng):
    from oracle.mps import two_site_mask
    mask = two_site_mask(ql, qr)
    return np.where(mask, rng.standard_normal(mask.shape), 0.0)


def require_gpu():
    if not gpu_available():
        pytest.skip("needs a CUDA device")
    library()
