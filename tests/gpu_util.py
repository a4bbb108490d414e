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


def check_product(kind: str, out: np.ndarray, u: np.ndarray, v: np.ndarray, n: int,
                  b: int = None, N: int = None, full=None) -> None:
    """Asserts that the limbs `out` are the oracle's product of kind for n-bit u, v:
    low and full bit for bit (Algorithms 1 and 2 are exact); high admissible
    (Section 1) and, when the plan (b, N) is given and n <= 2^18, equal to the exact
    round(t) of Algorithm 3 from the oracle's trace."""
    from oracle import trace
    if full is None:
        full = bigmul.mul_full(u, v, par_depth=3)
    nl = (n + 63) // 64
    if kind == "full":
        assert np.array_equal(out[: 2 * nl], full), f"full n={n}"
        return
    if kind == "lo":
        want = full[:nl].copy()
        if n % 64:
            want[-1] &= np.uint64((1 << (n % 64)) - 1)
        assert np.array_equal(out[:nl], want), f"low n={n}"
        return
    w = bigmul.to_int(out[: n // 64 + 1])
    assert hi_ok(w, u, v, n, full=full), f"high not admissible n={n}"
    if b is not None and N is not None and n <= 1 << 18:
        ex = trace.trace("hi", bigmul.to_int(u), bigmul.to_int(v), n, b, N)
        assert w == ex["out"], f"high round(t) n={n} b={b} N={N}"
