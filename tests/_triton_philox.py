"""Independent Philox4x32-10: Triton's own implementation run by its CPU
interpreter.  Reads JSON {"seeds": [...], "ctr": [[c0,c1,c2,c3], ...]} on
stdin and prints the 4 output words per (seed, counter) as JSON."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(c0p, c1p, c2p, c3p, outp, seed, n, BLOCK: tl.constexpr):
    offs = tl.arange(0, BLOCK)
    m = offs < n
    c0 = tl.load(c0p + offs, mask=m).to(tl.uint32, bitcast=True)
    c1 = tl.load(c1p + offs, mask=m).to(tl.uint32, bitcast=True)
    c2 = tl.load(c2p + offs, mask=m).to(tl.uint32, bitcast=True)
    c3 = tl.load(c3p + offs, mask=m).to(tl.uint32, bitcast=True)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(outp + offs * 4 + 0, a.to(tl.int32, bitcast=True), mask=m)
    tl.store(outp + offs * 4 + 1, b.to(tl.int32, bitcast=True), mask=m)
    tl.store(outp + offs * 4 + 2, c.to(tl.int32, bitcast=True), mask=m)
    tl.store(outp + offs * 4 + 3, d.to(tl.int32, bitcast=True), mask=m)


def main():
    req = json.load(sys.stdin)
    ctr = np.asarray(req["ctr"], np.uint64).astype(np.uint32)
    n = ctr.shape[0]
    block = 1 << max(0, (n - 1).bit_length())
    cols = [torch.from_numpy(ctr[:, j].view(np.int32).copy()) for j in range(4)]
    res = {}
    for s in req["seeds"]:
        out = torch.zeros(n * 4, dtype=torch.int32)
        _philox_kernel[(1,)](cols[0], cols[1], cols[2], cols[3], out, int(s), n, BLOCK=block)
        res[str(s)] = (out.numpy().view(np.uint32).reshape(n, 4)).tolist()
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
