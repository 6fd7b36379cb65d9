"""Small, fixed cases of the library's kernels for profilers (ncu) and timelines.

    python -m paper_2105_07076_gb300.profile_cases rid_small     # randomized ID, 4096 x 32768, k = 512
    python -m paper_2105_07076_gb300.profile_cases id_small      # deterministic ID, 2048 x 8192, k = 256, FP64
    python -m paper_2105_07076_gb300.profile_cases rid_timeline  # per-step phase times of the sketch's CPQR

rid_small runs the randomized ID on a matrix with 4096 rows instead of the
workload's 16384: the sketch (522 x 32768), its CPQR, the solve and the
refinement's products have the workload's shapes in every dimension but m, and
the device holds about 1.5 GB, so a multi-pass ncu capture of one kernel ends
quickly. Each case runs three warm-up calls, then `--reps` calls (default 1).
rid_timeline prints the sketch CPQR's mean phase times (microseconds) from the
library's step timeline (id_cpqr_timeline) on the full 16384 x 32768 workload.
"""
from __future__ import annotations

import argparse
import json


def _rid(m, reps, timeline=False):
    import torch

    import paper_2105_07076_gb300 as gbid
    import synth

    n, k, l = 32768, 512, 522
    dev = torch.device("cuda")
    A = synth.lowrank(m, n, synth.spectrum("poly1.5", m), 3, device=dev, dtype=torch.float32,
                      gen_dtype=torch.float32)
    om = synth.gaussian_sketch_bf16(l, m, seed=33, device=dev)
    ws = gbid.rid_workspace(m, n, l, k, device=dev)
    J = torch.empty(k, dtype=torch.int32, device=dev)
    Z = torch.empty(k, n, dtype=torch.float32, device=dev)
    for _ in range(3):
        gbid.id_decompose_randomized(A, om, k, workspace=ws, out=(J, Z), sync=False)
    tl = None
    if timeline:
        tl = torch.zeros(k * 8, dtype=torch.int64, device=dev)
        gbid.cpqr_timeline(tl)
    for _ in range(reps):
        gbid.id_decompose_randomized(A, om, k, workspace=ws, out=(J, Z), sync=False)
    torch.cuda.synchronize()
    if timeline:
        gbid.cpqr_timeline(None)
        t = tl.view(k, 8).cpu().double()
        d = (t[:, 1:6] - t[:, 0:5]) / 1e3
        names = ["pivot", "column", "reflector_aux", "product", "barrier"]
        out = {}
        for lo, hi in ((0, 32), (32, 256), (256, 512), (0, 512)):
            out[f"steps {lo}-{hi - 1}"] = dict({nm: round(d[lo:hi, i].mean().item(), 2) for i, nm in enumerate(names)},
                                              step=round(((t[lo:hi, 5] - t[lo:hi, 0]) / 1e3).mean().item(), 2))
        out["between_steps_ms"] = round(((t[1:, 0] - t[:-1, 5]).sum() / 1e6).item(), 3)
        out["steps_ms"] = round(((t[:, 5] - t[:, 0]).sum() / 1e6).item(), 3)
        print(json.dumps(out))
    print(json.dumps(gbid.read_info(ws)))


def _id(reps):
    import torch

    import paper_2105_07076_gb300 as gbid
    import synth

    m, n, k = 2048, 8192, 256
    A = synth.lowrank(m, n, synth.spectrum("exp64", m), 2, device="cuda")
    ws = gbid.Workspace.for_problem(A.dtype, m, n, k, device="cuda")
    J = torch.empty(k, dtype=torch.int32, device="cuda")
    Z = torch.empty(k, n, dtype=A.dtype, device="cuda")
    for _ in range(3 + reps):
        gbid.id_decompose(A, k, workspace=ws, out=(J, Z), sync=False)
    torch.cuda.synchronize()
    print(json.dumps(gbid.read_info(ws)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["rid_small", "id_small", "rid_timeline"])
    ap.add_argument("--reps", type=int, default=1)
    args = ap.parse_args()
    import __graft_entry__ as ge

    ge.build()
    if args.case == "rid_small":
        _rid(4096, args.reps)
    elif args.case == "rid_timeline":
        _rid(16384, 1, timeline=True)
    else:
        _id(args.reps)


if __name__ == "__main__":
    main()
