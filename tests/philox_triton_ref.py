"""Philox-4x32-R words from Triton's own implementation (triton.language.philox), run by Triton's
CPU interpreter: an implementation of Salmon et al.'s generator (SC'11) written independently of
this repository, used only to pin the oracle's 4x32 instance.

Run as a script with TRITON_INTERPRET=1 in the environment (the interpreter must be chosen before
any kernel is defined, so the caller starts a fresh process): reads one JSON object
{"rounds": R, "cases": [[k0, k1, [[c0, c1, c2, c3], ...]], ...]} on stdin and prints the words,
one list of [w0, w1, w2, w3] per case, as JSON. Triton takes the key as one 64-bit seed whose low
half is k0 and high half k1.
"""
import json
import sys


def main():
    import numpy as np
    import torch
    import triton
    import triton.language as tl

    @triton.jit
    def words(c0p, c1p, c2p, c3p, seed, o0, o1, o2, o3, N: tl.constexpr, R: tl.constexpr):
        i = tl.arange(0, N)
        a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i),
                               tl.load(c3p + i), R)
        tl.store(o0 + i, a)
        tl.store(o1 + i, b)
        tl.store(o2 + i, c)
        tl.store(o3 + i, d)

    req = json.load(sys.stdin)
    out = []
    for k0, k1, ctrs in req["cases"]:
        c = np.asarray(ctrs, dtype=np.uint64).reshape(-1, 4).astype(np.uint32)
        n = c.shape[0]
        npow = 1 << max(0, (n - 1).bit_length())
        cp = np.zeros((npow, 4), np.uint32)
        cp[:n] = c
        ins = [torch.from_numpy(np.ascontiguousarray(cp[:, w]).view(np.int32)) for w in range(4)]
        outs = [torch.empty(npow, dtype=torch.int32) for _ in range(4)]
        words[(1,)](*ins, (int(k1) << 32) | int(k0), *outs, N=npow, R=int(req["rounds"]))
        w = np.stack([o.numpy().view(np.uint32) for o in outs], axis=1)[:n]
        out.append(w.astype(np.int64).tolist())
    json.dump(out, sys.stdout)


if __name__ == "__main__":
    main()
