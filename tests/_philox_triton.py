"""Run Triton's own Philox4x32-10 (triton.language.philox, Python source) on
the CPU through the Triton interpreter, for counters and keys given on stdin
as JSON; print its four output words per input.  Used only as an independent
known-answer source for the oracle's generator."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kernel(c0p, c1p, c2p, c3p, o0, o1, o2, o3, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(o0 + i, a)
    tl.store(o1 + i, b)
    tl.store(o2 + i, c)
    tl.store(o3 + i, d)


def main():
    req = json.load(sys.stdin)
    out = []
    for seed, ctrs in req:
        ctr = np.array(ctrs, dtype=np.uint32).reshape(-1, 4)
        n = ctr.shape[0]
        cols = [torch.from_numpy(ctr[:, j].astype(np.int64)).to(torch.uint32) for j in range(4)]
        outs = [torch.zeros(n, dtype=torch.uint32) for _ in range(4)]
        _kernel[(1,)](*cols, *outs, seed, n)
        out.append(np.stack([o.to(torch.int64).numpy() for o in outs], axis=1).tolist())
    json.dump(out, sys.stdout)


if __name__ == "__main__":
    main()
