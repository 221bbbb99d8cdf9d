"""Independent Philox4x32-10 outputs from Triton's own implementation.

Run as a script with TRITON_INTERPRET=1 (Triton's CPU interpreter), it reads
JSON {"ctr": [[c0,c1,c2,c3], ...], "seed": [s, ...]} on stdin and prints
JSON [[o0,o1,o2,o3], ...] on stdout.  Triton's ``tl.philox(seed, c0..c3)``
uses key (seed mod 2^32, seed >> 32) for 32-bit counters, the same key
convention as the oracle.  This is a third-party implementation used only to
pin the oracle's Philox; it is not part of the product.
"""
import json
import os
import sys


def main():
    os.environ["TRITON_INTERPRET"] = "1"
    import torch
    import triton
    import triton.language as tl

    @triton.jit
    def philox_kernel(out_ptr, c_ptr, seed_ptr, n, BLOCK: tl.constexpr):
        i = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c_ptr + 4 * i + 0, mask=m)
        c1 = tl.load(c_ptr + 4 * i + 1, mask=m)
        c2 = tl.load(c_ptr + 4 * i + 2, mask=m)
        c3 = tl.load(c_ptr + 4 * i + 3, mask=m)
        seed = tl.load(seed_ptr + i, mask=m)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a, mask=m)
        tl.store(out_ptr + 4 * i + 1, b, mask=m)
        tl.store(out_ptr + 4 * i + 2, c, mask=m)
        tl.store(out_ptr + 4 * i + 3, d, mask=m)

    req = json.load(sys.stdin)
    n = len(req["ctr"])
    ctr = torch.tensor([v for row in req["ctr"] for v in row],
                       dtype=torch.int64).to(torch.uint32)
    seed = torch.tensor([s if s < 2 ** 63 else s - 2 ** 64 for s in req["seed"]],
                        dtype=torch.int64)
    out = torch.zeros(4 * n, dtype=torch.uint32)
    BLOCK = 64
    philox_kernel[((n + BLOCK - 1) // BLOCK,)](out, ctr, seed, n, BLOCK=BLOCK)
    vals = out.to(torch.int64) & 0xFFFFFFFF
    res = vals.view(n, 4).tolist()
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
