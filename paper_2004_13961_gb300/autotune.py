"""Tune the tile shapes of the FP64 K x contractions on this GPU and write the table
the library compiles in (csrc/xf_tiles_gb300.inc).

    python -m paper_2004_13961_gb300.autotune [--out PATH] [--reps R]

The sizes are those of the workloads: the batched 2D problems N = 32, 48, ..., 256
(Q = N + 2, T = 8), the 2D N = 64 and N = 512 problems, and the 3D N = 64 and 128
problems.  Each entry is the choice lsg_autotune_transforms makes on a context of
that size (coefficients a = b = 1: the contraction times do not depend on values).
Rebuild the library afterwards (build.py) so that new contexts start with the table.
"""
from __future__ import annotations

import argparse
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

SIZES = [(2, N) for N in range(32, 257, 16)] + [(2, 512), (3, 64), (3, 128)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "csrc", "xf_tiles_gb300.inc"))
    ap.add_argument("--reps", type=int, default=10)
    args = ap.parse_args()
    import torch
    from . import lsg
    lsg.load()
    dev = torch.device("cuda", 0)
    rows = []
    for d, N in SIZES:
        Q = N + 2
        T = 0  # the contractions do not depend on T; the narrowest stencil keeps setup cheap
        ones = torch.ones(Q ** d, dtype=torch.float64, device=dev)
        ctx = lsg.Context(d, N, T, ones, ones, Q=Q)
        default = ctx.transform_tiles()
        x = torch.randn(ctx.n, dtype=torch.float64, device=dev)
        y = torch.empty_like(x)

        def t_kx(reps=20):
            ctx.apply_A(x, y)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            for _ in range(reps):
                ctx.apply_A(x, y)
            e.record()
            torch.cuda.synchronize()
            return s.elapsed_time(e) / reps

        t_def = t_kx()
        choice = ctx.autotune_transforms(args.reps)
        t_best = t_kx()
        rows.append((d, N, Q, choice[:3], choice[3:]))
        print(f"d={d} N={N}: default {default} {t_def * 1e3:.1f} us -> {choice} {t_best * 1e3:.1f} us", flush=True)
        ctx.close()
    with open(args.out, "w") as fh:
        fh.write("// Tile variants of the FP64 contractions chosen by the autotuner on a GB300:\n"
                 "// {d, N, Q, {forward contraction 1..d}, {backward contraction 1..d}}, variant\n"
                 "// indices of transform.cu (0: 16x16, 1: 16x32, 2: 32x32, 3: 32x64, 4: 64x32;\n"
                 "// -1: the default).  Written by paper_2004_13961_gb300/autotune.py.\n")
        for d, N, Q, f, b in rows:
            fh.write("{%d, %d, %d, {%d, %d, %d}, {%d, %d, %d}},\n" % (d, N, Q, *f, *b))
    print("wrote", args.out)


if __name__ == "__main__":
    main()
