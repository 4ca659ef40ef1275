"""The library has no CPU path and no silent fallback: host tensors are refused
before any call, and a missing CUDA toolchain stops the build with an error
instead of substituting anything.  No GPU needed."""
import pytest
import torch

import paper_2212_06985_gb300 as t3d
from paper_2212_06985_gb300 import build as build_mod


def test_host_tensors_are_refused():
    e = torch.zeros((3 * 4 ** 3, 1), dtype=torch.int64)
    with pytest.raises(ValueError, match="no CPU path"):
        t3d.toric3d_noise(4, e, 0.1, 0, 0, 1)


def test_missing_nvcc_is_an_error(monkeypatch):
    monkeypatch.setenv("NVCC", "/nonexistent/nvcc")
    monkeypatch.setattr(build_mod.shutil, "which", lambda name: None)
    real_exists = build_mod.os.path.exists
    monkeypatch.setattr(build_mod.os.path, "exists",
                        lambda p: False if str(p).endswith("nvcc") else real_exists(p))
    with pytest.raises(RuntimeError, match="nvcc not found"):
        build_mod._nvcc()
