"""Helpers shared by the GPU tests (device transfer only, no field arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch.device("cuda:0")


def to_dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def to_host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def device_bytes(n: int, seed: int):
    """Seeded uniform bytes generated on the device (for sizes the host
    should not generate); the oracle receives the same bytes by copying the
    sampled inputs back."""
    g = torch.Generator(device=dev())
    g.manual_seed(seed)
    return torch.randint(0, 256, (n,), dtype=torch.uint8, device=dev(), generator=g)
