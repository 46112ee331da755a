"""Profiling driver: a fixed number of solves of the 4K RGB bench workload
through the public API, for capturing kernels with ncu.

  python -m paper_2401_06747_b300.prof_case --kind inpaint --solves 2
"""

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", choices=["inpaint", "tonal"], default="inpaint")
    ap.add_argument("--solves", type=int, default=2)
    ap.add_argument("--height", type=int, default=2160)
    ap.add_argument("--width", type=int, default=3840)
    a = ap.parse_args()
    import numpy as np
    import torch
    import paper_2401_06747_b300 as hdi
    from synthdata import synth_rgb, random_mask
    f = synth_rgb(a.height, a.width, seeds=(1, 2, 3), dtype=np.float32)
    c = random_mask(a.height, a.width, 0.04, 1001)
    ctx = hdi.Context(0)
    fd = torch.from_numpy(f).cuda()
    cd = torch.from_numpy(c).cuda()
    out = torch.empty_like(fd)
    for _ in range(a.solves):
        st = ctx.inpaint(fd, cd, out, tol=1e-6) if a.kind == "inpaint" else ctx.tonal_opt(fd, cd, out, tol=1e-6)
    torch.cuda.synchronize()
    print(st)


if __name__ == "__main__":
    main()
