"""Print Philox4x32-10 outputs computed by Triton's own implementation (interpreter mode).

Each output line: c0 c1 c2 c3 k0 k1 r0 r1 r2 r3. Exit code 77 when the interpreter
cannot run here.
"""
import os
import sys

os.environ.setdefault("TRITON_INTERPRET", "1")
try:
    import numpy as np
    import torch
    import triton
    import triton.language as tl
except Exception as exc:  # pragma: no cover
    print(exc)
    sys.exit(77)


@triton.jit
def _philox_kernel(c0p, c1p, c2p, c3p, k0p, k1p, o0, o1, o2, o3, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c0p + i)
    c1 = tl.load(c1p + i)
    c2 = tl.load(c2p + i)
    c3 = tl.load(c3p + i)
    k0 = tl.load(k0p + i)
    k1 = tl.load(k1p + i)
    r0, r1, r2, r3 = tl.philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(o0 + i, r0)
    tl.store(o1 + i, r1)
    tl.store(o2 + i, r2)
    tl.store(o3 + i, r3)


def main():
    n = 64
    g = np.random.default_rng(2024)
    vals = g.integers(0, 2 ** 32, size=(6, n), dtype=np.uint64)
    vals[:, 0] = 0
    vals[:, 1] = 0xFFFFFFFF
    ins = [torch.from_numpy(v.astype(np.uint32).view(np.int32).copy()).view(torch.uint32) for v in vals]
    outs = [torch.zeros(n, dtype=torch.uint32) for _ in range(4)]
    try:
        _philox_kernel[(1,)](*ins, *outs, N=n)
    except Exception as exc:  # pragma: no cover
        print(exc)
        sys.exit(77)
    res = [o.view(torch.int32).numpy().view(np.uint32).astype(np.uint64) for o in outs]
    for r in range(n):
        print(" ".join(str(int(x)) for x in list(vals[:, r]) + [res[c][r] for c in range(4)]))


if __name__ == "__main__":
    main()
