"""Philox4x32-10 computed by Triton's own implementation, run on the CPU.

Executed in a subprocess with TRITON_INTERPRET=1 (Triton's interpreter runs the
kernel with numpy).  Reads JSON [[c0, c1, c2, c3, k0, k1], ...] on stdin and
prints the four output words of each row as JSON.
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(c_ptr, k_ptr, o_ptr, n, BLOCK: tl.constexpr):
    offs = tl.arange(0, BLOCK)
    m = offs < n
    c0 = tl.load(c_ptr + offs * 4 + 0, mask=m, other=0)
    c1 = tl.load(c_ptr + offs * 4 + 1, mask=m, other=0)
    c2 = tl.load(c_ptr + offs * 4 + 2, mask=m, other=0)
    c3 = tl.load(c_ptr + offs * 4 + 3, mask=m, other=0)
    k0 = tl.load(k_ptr + offs * 2 + 0, mask=m, other=0)
    k1 = tl.load(k_ptr + offs * 2 + 1, mask=m, other=0)
    a, b, c, d = tl.philox_impl(c0, c1, c2, c3, k0, k1)
    tl.store(o_ptr + offs * 4 + 0, a, mask=m)
    tl.store(o_ptr + offs * 4 + 1, b, mask=m)
    tl.store(o_ptr + offs * 4 + 2, c, mask=m)
    tl.store(o_ptr + offs * 4 + 3, d, mask=m)


def main():
    rows = np.array(json.load(sys.stdin), dtype=np.uint64).reshape(-1, 6)
    n = rows.shape[0]
    block = 1
    while block < n:
        block *= 2
    c = torch.from_numpy(rows[:, :4].astype(np.uint32).view(np.int32).copy())
    k = torch.from_numpy(rows[:, 4:].astype(np.uint32).view(np.int32).copy())
    c = c.view(torch.uint32) if hasattr(torch, "uint32") else c
    k = k.view(torch.uint32) if hasattr(torch, "uint32") else k
    o = torch.zeros((n, 4), dtype=c.dtype)
    _philox_kernel[(1,)](c, k, o, n, BLOCK=block)
    out = o.view(torch.int32).numpy().view(np.uint32).astype(np.int64).tolist()
    json.dump(out, sys.stdout)


if __name__ == "__main__":
    main()
