"""Small, bounded cases of the library's kernels for profiling (ncu).

    python -m paper_2105_05879_gb300.profile_cases <case> [--reps R]

Cases hold a few GB on the device at most and run each kernel R + 2 times
(two warm-up launches), so a profiler can skip the warm-up launches and
capture one or two launches that end by themselves.
  pre4096   kerdock_preprocess, m = 256, n = 4096, bfloat16 (4.3 GB)
  q4096     kerdock_apply, m = 256, n = 4096, bfloat16, 512 queries, J = 1000, K = 2
  pre1024   kerdock_preprocess, m = n = 1024, float32 (2.15 GB)
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["pre4096", "q4096", "pre1024"])
    ap.add_argument("--reps", type=int, default=1)
    args = ap.parse_args()
    import torch
    from paper_2105_05879_gb300 import build as kbuild
    from paper_2105_05879_gb300 import kerdock as K
    kbuild.build()
    K.load_library()
    torch.manual_seed(0)
    if args.case == "pre1024":
        m = n = 1024
        dtype = "f32"
    else:
        m, n, dtype = 256, 4096, "bf16"
    A = (torch.randn(m, n, device="cuda") / n ** 0.5).contiguous()
    plan = K.KerdockPlan(m, n, J=1000, K=2, S=32, dtype=dtype)
    if args.case in ("pre4096", "pre1024"):
        for _ in range(args.reps + 2):
            plan.preprocess(A)
    else:
        plan.preprocess(A)
        X = torch.randn(512, n, device="cuda")
        X /= X.norm(dim=1, keepdim=True)
        for _ in range(args.reps + 2):
            plan.apply(X, 0.1, 3)
    plan.sync()
    torch.cuda.synchronize()
    print("ok", args.case)


if __name__ == "__main__":
    main()
