"""Both Wick topologies of a baryon with two identical spectator flavours from one
spectator call: the exchange topology is the spectator with the two quark lines' indices
permuted, which the combine takes as W_snk and W_src with their first two indices
transposed.  Against the oracle's combine of the spectator with the propagators swapped."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS
from oracle import contractions as OC

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_exchange_topology_by_index_permutation(prec, tol):
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import lhc
    c = CS.Case(3, 4, 3, momenta(2), seed=2300, r=(0, 1, 2, 0))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ws = CS.random_gammas(2301, 2, (4, 4, 4))
    wc = CS.random_gammas(2302, 2, (4, 4, 4))
    gi = CS.random_gammas(2303, 2, (4, 4))
    t = 2
    with lhc.Context(0) as ctx:
        B = ctx.spectator(dev(c.S), dev(c.eta(t)), t, c.r, c.k, prec=prec, GB=dev(c.SB))
        ins = ctx.insertion(dev(c.S), dev(c.psi), 1, 1, c.r, c.k, prec=prec)[0]
        direct = ctx.combine(B, ins, dev(ws), dev(gi), dev(wc), prec=prec).cpu().numpy()
        exch = ctx.combine(B, ins, dev(ws.transpose(0, 2, 1, 3)), dev(gi), dev(wc.transpose(0, 2, 1, 3)),
                           prec=prec).cpu().numpy()
        ctx.sync()
    g5 = CS.g5_matrix()
    I_ref = c.ref_insertion(1, 1)[0]
    B_ab = OC.spectator_baryon(c.S[t], c.SB[t], c.eta(t), g5, c.r[:3], c.k, c.L)
    B_ba = OC.spectator_baryon(c.SB[t], c.S[t], c.eta(t), g5, c.r[:3], c.k, c.L)   # quark lines exchanged
    assert CS.corr_err(direct, OC.combine_baryon(B_ab, I_ref, ws, gi, wc)) < tol
    assert CS.corr_err(exch, OC.combine_baryon(B_ba, I_ref, ws, gi, wc)) < tol
