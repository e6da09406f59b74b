"""Device transfer helpers for the GPU tests (uint32 words via int32 tensors)."""
import numpy as np
import torch


def to_dev(a: np.ndarray, pad: int = 0) -> torch.Tensor:
    """Copy a uint32 matrix to the GPU; with pad > 0 the rows get extra columns
    (a larger leading dimension) and the returned view has the original shape."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    if pad:
        buf = np.zeros((a.shape[0], a.shape[1] + pad), np.uint32)
        buf[:, : a.shape[1]] = a
        t = torch.from_numpy(buf.view(np.int32)).cuda()
        return t[:, : a.shape[1]]
    return torch.from_numpy(a.view(np.int32)).cuda()


def from_dev(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().cpu().numpy().view(np.uint32)
