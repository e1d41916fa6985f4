"""Run one kernel configuration a few times, for profiling with ncu.

    python -m paper_1711_02384_gb300.profile_case --part ins --L 24 --nr 16 --n2max 8 \
        --slices 2 --reps 3 --prec mixed --dtype c128

Inputs are random device tensors (torch, seeded): this driver only exercises the
kernels; parity is the tests' job.  Prints the CUDA-event time per call.
"""
import argparse
import json

import torch

from . import lhc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--part", choices=["ins", "spec", "baryon", "combine"], default="ins")
    ap.add_argument("--L", type=int, default=24)
    ap.add_argument("--nr", type=int, default=16)
    ap.add_argument("--n2max", type=int, default=8)
    ap.add_argument("--slices", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--dtype", choices=["c128", "c64"], default="c128")
    ap.add_argument("--gammas", choices=["random", "sweep"], default="random",
                    help="combine: 16 random structures everywhere, or the Dirac sweep at sink "
                         "and source with gamma_4 at the insertion (the benchmark's)")
    a = ap.parse_args()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(1234)
    dt = torch.complex128 if a.dtype == "c128" else torch.complex64
    V3 = a.L ** 3
    k = lhc.momenta(a.n2max)
    r = (0, 0, 0, 0)
    T = a.slices
    S = torch.randn((T, V3, 12, 12), dtype=dt, device=dev, generator=g)
    ctx = lhc.Context(0)
    if a.part == "ins":
        psi = torch.randn((a.nr, T, V3, 12), dtype=dt, device=dev, generator=g)
        call = lambda: ctx.insertion(S, psi, 0, T - 1, r, k, prec=a.prec)
    elif a.part in ("spec", "baryon"):
        eta = torch.randn((a.nr, V3, 12), dtype=dt, device=dev, generator=g)
        GB = torch.randn((T, V3, 12, 12), dtype=dt, device=dev, generator=g) if a.part == "baryon" else None
        call = lambda: ctx.spectator(S, eta, 0, r, k, prec=a.prec, GB=GB)
    else:
        nq = len(k)
        spec = torch.randn((nq, a.nr, 192), dtype=torch.complex128, device=dev, generator=g)
        ins = torch.randn((T, nq, a.nr, 192), dtype=torch.complex128, device=dev, generator=g)
        if a.gammas == "sweep":
            from . import inputs
            G = torch.from_numpy(inputs.dirac_structures()).to(dev)
            Gi = torch.from_numpy(inputs.dirac_matrices()[3]).to(dev).expand(16, 4, 4).contiguous()
        else:
            G = Gi = torch.randn((16, 4, 4), dtype=torch.complex128, device=dev, generator=g)
        call = lambda: ctx.combine(spec, ins, G, Gi, G, prec=a.prec)
    call()
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        call()
    e1.record()
    ctx.sync()
    print(json.dumps({"case": vars(a), "ms_per_call": e0.elapsed_time(e1) / a.reps}))
    ctx.close()


if __name__ == "__main__":
    main()
