"""Helpers for the GPU tests: numpy <-> torch limb tensors and oracle checks."""
import numpy as np
import torch

from oracle import bigmul


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def hi_ok(w: int, u: np.ndarray, v: np.ndarray, n: int, full=None) -> bool:
    """w is an admissible high product (Section 1)."""
    if full is None:
        q, nz = bigmul.mul_hi_floor(u, v, n, par_depth=3)
        q = bigmul.to_int(q)
    else:
        uv = bigmul.to_int(full)
        q, nz = uv >> n, (uv & ((1 << n) - 1)) != 0
    return w == q or (nz and w == q + 1)
