"""Fused kernels of different calls running at the same time: four contexts, each on its
own stream (a context orders its own calls, so concurrency needs several), issue
insertions, meson spectators and baryon spectators of several lattices and momentum
chunk widths round-robin with no synchronization between them.  Every result equals the
same call made alone, bit for bit, and the library's error word stays clear.  This is
the launch pattern of the job server's slots."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_concurrent_fused_launches_equal_calls_alone():
    from paper_1711_02384_gb300 import lhc
    # (L, T, n_r, |k|^2 max): 147 momenta give chunks of 40, 93 of 48, 33 of 24
    shapes = [(12, 8, 16, 10), (10, 8, 8, 8), (16, 8, 16, 4), (8, 8, 32, 10)]
    cases = [CS.Case(L, T, n_r, lhc.momenta(n2), seed=2700 + 10 * i, dtype=np.complex64)
             for i, (L, T, n_r, n2) in enumerate(shapes)]
    data = [(dev(c.S), dev(c.SB), dev(c.psi), dev(c.eta(3))) for c in cases]

    def calls(ctx, i, st):
        c = cases[i]
        S, SB, psi, eta = data[i]
        s = st.cuda_stream
        return [ctx.insertion(S, psi, 0, 5, c.r, c.k, stream=s),
                ctx.spectator(S, eta, 3, c.r, c.k, stream=s),
                ctx.spectator(S, eta, 3, c.r, c.k, GB=SB, stream=s)]

    ctxs = [lhc.Context(0) for _ in cases]
    streams = [torch.cuda.Stream() for _ in cases]
    try:
        for x in ctxs:
            x.set_projection("gemm")
        alone = []
        for i, (x, st) in enumerate(zip(ctxs, streams)):
            alone.append(calls(x, i, st))
            st.synchronize()
            x.sync(st.cuda_stream)
        rounds = []
        for _ in range(3):
            rounds.append([calls(x, i, st) for i, (x, st) in enumerate(zip(ctxs, streams))])
        for i, (x, st) in enumerate(zip(ctxs, streams)):
            st.synchronize()
            x.sync(st.cuda_stream)
        for got in rounds:
            for i in range(len(cases)):
                for a, b in zip(got[i], alone[i]):
                    assert torch.equal(a, b), f"case {i} differs when run beside the others"
    finally:
        for x in ctxs:
            x.close()
    c = cases[0]
    assert CS.block_err(alone[0][0].cpu().numpy(), c.ref_insertion(0, 5), 2) < CS.MIXED_TOL
