"""Philox4x32-10 computed by Triton's own implementation (triton.language.random
.philox_impl) through Triton's CPU interpreter.  Used as an independent,
third-party pin for the oracle's Philox.  Run as a script in a fresh process
(TRITON_INTERPRET must be set before triton is imported):

    python tests/_triton_philox.py in.npy out.npy k0 k1
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402
from triton.language.random import philox_impl  # noqa: E402


@triton.jit
def _kernel(c0p, c1p, c2p, c3p, o0, o1, o2, o3, k0, k1, n, BLOCK: tl.constexpr):
    i = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    m = i < n
    c0 = tl.load(c0p + i, mask=m).to(tl.uint32)
    c1 = tl.load(c1p + i, mask=m).to(tl.uint32)
    c2 = tl.load(c2p + i, mask=m).to(tl.uint32)
    c3 = tl.load(c3p + i, mask=m).to(tl.uint32)
    kk0 = tl.full((BLOCK,), k0, tl.uint32)
    kk1 = tl.full((BLOCK,), k1, tl.uint32)
    a, b, c, d = philox_impl(c0, c1, c2, c3, kk0, kk1)
    tl.store(o0 + i, a, mask=m)
    tl.store(o1 + i, b, mask=m)
    tl.store(o2 + i, c, mask=m)
    tl.store(o3 + i, d, mask=m)


def main():
    ctr = np.load(sys.argv[1]).astype(np.uint32).reshape(-1, 4)
    k0, k1 = int(sys.argv[3]), int(sys.argv[4])
    n = ctr.shape[0]
    C = [torch.from_numpy(np.ascontiguousarray(ctr[:, j])) for j in range(4)]
    O = [torch.from_numpy(np.zeros(n, np.uint32)) for _ in range(4)]
    BLOCK = 1024
    _kernel[(triton.cdiv(n, BLOCK),)](*C, *O, np.uint32(k0), np.uint32(k1), n, BLOCK=BLOCK)
    np.save(sys.argv[2], np.stack([o.numpy() for o in O], axis=1))


if __name__ == "__main__":
    main()
