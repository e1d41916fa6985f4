"""Batched calls (lhc_batch): many mixed-precision insertion and spectator calls with
uneven momentum sets, lattices and parts in one fused launch per part kind; the results
must equal, bit for bit, those of the same calls made one by one with the tensor-core
projection, and one of them the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


def test_batch_equals_single_calls():
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import lhc
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cases = [CS.Case(4, 8, 2, momenta(2), seed=2500, r=(1, 2, 3, 0)),
             CS.Case(6, 6, 3, momenta(5), seed=2501, r=(0, 4, 1, 0), dtype=np.complex64),
             CS.Case(5, 4, 2, momenta(9, 3), seed=2502, r=(2, 2, 2, 0))]
    calls = []
    for n, c in enumerate(cases):
        S, SB, psi = dev(c.S), dev(c.SB), dev(c.psi)
        eta = dev(c.eta(2))
        t_lo = [1, 4, 0][n]                                      # the second range wraps around T = 6
        calls.append(dict(part="ins", S=S, vec=psi, t_lo=t_lo, t_hi=t_lo + 2, r=c.r, k=c.k))
        calls.append(dict(part="spec", S=S, vec=eta, t_lo=2, t_hi=2, r=c.r, k=c.k))
        calls.append(dict(part="baryon", S=S, GB=SB, vec=eta, t_lo=2, t_hi=2, r=c.r, k=c.k))
    with lhc.Context(0) as ctx:
        got = ctx.batch(calls)
        auto = ctx.insertion(calls[6]["S"], calls[6]["vec"], 0, 2, cases[2].r, cases[2].k, prec="mixed")
        ctx.set_projection("gemm")                               # the batch always projects on the tensor cores
        ref = []
        for c in calls:
            if c["part"] == "ins":
                ref.append(ctx.insertion(c["S"], c["vec"], c["t_lo"], c["t_hi"], c["r"], c["k"], prec="mixed"))
            else:
                ref.append(ctx.spectator(c["S"], c["vec"], c["t_lo"], c["r"], c["k"], prec="mixed", GB=c.get("GB")))
        again = ctx.batch(calls)                                 # a second batch reproduces the first
        ctx.sync()
    for g, r, a in zip(got, ref, again):
        assert torch.equal(g, r)
        assert torch.equal(g, a)
    # the third case asks for every momentum, so the same call made alone takes the
    # all-momenta transform: another rounding order, within the mixed tolerance
    assert CS.block_err(auto.cpu().numpy(), got[6].cpu().numpy(), 2) < CS.MIXED_TOL
    c = cases[0]
    assert CS.block_err(got[0].cpu().numpy(), c.ref_insertion(1, 3), 2) < CS.MIXED_TOL
    assert CS.block_err(got[2].cpu().numpy(), c.ref_spectator_baryon(2), 1) < CS.MIXED_TOL
