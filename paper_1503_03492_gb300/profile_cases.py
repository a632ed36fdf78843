"""Small, fixed workloads for profiling the kernels (e.g. under ncu).

    python -m paper_1503_03492_gb300.profile_cases standard512 [--cycles 20]
        one standard projection (persistent kernel) of the 512 x 512 emitter
        residual, window sides 1..8, a fixed number of cycles;
    python -m paper_1503_03492_gb300.profile_cases icd512
        one incomplete projection (K = 3, tol 1e-3) of the same image;
    python -m paper_1503_03492_gb300.profile_cases batch512 [--images 8] [--q fp32|bf16|fp16] [--cycles 3]
        a batch of copies of that image (one step-kernel launch per group);
    python -m paper_1503_03492_gb300.profile_cases uneven [--images 32] [--q bf16] [--cycles 2]
        the first images of the uneven 256-image batch (sides 128..1024, half 2:1);
    python -m paper_1503_03492_gb300.profile_cases img2048 [--q bf16] [--cycles 2] [--per-side]
        the 2048 x 2048 emitter residual with window sides 1..12 (batched path;
        --per-side: one cooperative launch per side, SMRE_BF_PER_SIDE);
    python -m paper_1503_03492_gb300.profile_cases admm512 [--iters 3] [--cycles 20]
        the ADMM outer loop on the same image (PSF sigma 2, 20 TV steps per
        iteration, a fixed number of projection cycles per eps-step).

Each prints the device time it measured.  Inputs are the seeded synthetic
images of ``synthetic``; nothing is timed that the library does not run.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

QTYPES = {"fp32": 0, "bf16": 1, "fp16": 2}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["standard512", "icd512", "batch512", "uneven", "img2048", "admm512"])
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--cycles", type=int, default=None)
    ap.add_argument("--images", type=int, default=None)
    ap.add_argument("--q", choices=list(QTYPES), default="fp32")
    ap.add_argument("--per-side", action="store_true")
    a = ap.parse_args(argv)

    import torch
    import paper_1503_03492_gb300 as smre
    from synthetic import batch_images, emitter_residual, emitter_residual_2048

    torch.cuda.set_device(0)
    sides = list(range(1, 9))
    cS = smre.smre_bounds(smre.make_params(64, 64, sides))
    x0 = np.ascontiguousarray(emitter_residual(), np.float32)
    if a.case in ("standard512", "icd512"):
        xd = torch.from_numpy(x0).cuda()
        out = torch.empty_like(xd)
        with smre.Projector(512, 512, sides, cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS,
                            max_cycles=a.cycles or 20, tol=-1.0) as P:
            if a.case == "standard512":
                r = P.project(xd, out)
                print(f"standard512: {r.cycles} cycles, {r.seconds * 1e3:.3f} ms")
            else:
                r = P.project_incomplete(xd, out, K=3, tol=1e-3)
                print(f"icd512: {r.cycles} sweeps, {r.seconds * 1e3:.3f} ms")
        return 0
    if a.case == "admm512":
        I = torch.from_numpy(x0).cuda()
        x = torch.empty_like(I)
        with smre.Admm(512, 512, sides, 2.0, tv_iters=20, max_iters=a.iters, delta=-1.0,
                       cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS, max_cycles=a.cycles or 20,
                       tol=-1.0) as A:
            r = A.solve(I, x)
        print(f"admm512: {r.iters} iterations, {r.seconds * 1e3:.3f} ms "
              f"(projection {r.projection_seconds * 1e3:.3f} ms)")
        return 0
    if a.case == "batch512":
        xs = [torch.from_numpy(x0).cuda() for _ in range(a.images or 8)]
    elif a.case == "img2048":
        sides = list(range(1, 13))
        cS = smre.smre_bounds(smre.make_params(64, 64, sides))
        xs = [torch.from_numpy(np.ascontiguousarray(emitter_residual_2048(), np.float32)).cuda()]
    else:
        xs = [torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
              for x in batch_images(256)[: a.images or 32]]
    cycles = a.cycles or 3
    q = QTYPES[a.q]
    need = sum(smre.smre_batch_image_bytes(smre.make_batch_params(sides, q_dtype=q,
                                                                  max_cycles=cycles), *x.shape)
               for x in xs)
    with smre.Batch(sides, cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS, q_dtype=q,
                    flags=smre.SMRE_BF_PER_SIDE if a.per_side else 0,
                    max_cycles=cycles, tol=-1.0, max_images=len(xs),
                    device_bytes=need + (64 << 20)) as B:
        for x in xs:
            B.submit(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.run(cycles)
        e1.record()
        torch.cuda.synchronize()
        for s in B.poll():
            B.retrieve(s)
    print(f"{a.case}: {len(xs)} images, {cycles} cycles ({a.q}), {e0.elapsed_time(e1):.3f} ms")
    return 0


if __name__ == "__main__":
    sys.exit(main())
