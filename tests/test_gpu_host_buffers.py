"""Calls with host (pinned) buffers run asynchronously through the staging slots, with a
call's slices copied and computed in groups: a chain of insertion, spectator and combine
calls whose combine reads the host outputs of the calls before it must give, bit for
bit, the results of the same calls on device buffers; and one synchronize at the end
must suffice."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_chained_host_calls_match_device_calls(prec):
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import lhc
    c = CS.Case(6, 8, 3, momenta(2), seed=1900, r=(1, 0, 2, 0))
    G = CS.random_gammas(1901, 3, (4, 4))
    sets = [(1, 6, 6), (7, 10, 2)]           # (t_lo, t_hi, t_sink); the second wraps around T = 8
    with lhc.Context(0) as ctx:
        # device reference
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        ref = []
        for t_lo, t_hi, ts in sets:
            ins = ctx.insertion(dev(c.S), dev(c.psi), t_lo, t_hi, c.r, c.k, prec=prec)
            spec = ctx.spectator(dev(c.S), dev(c.eta(ts)), ts, c.r, c.k, prec=prec)
            comb = ctx.combine(spec, ins, dev(G), dev(G), dev(G), prec=prec)
            ref.append((ins.cpu(), spec.cpu(), comb.cpu()))
        ctx.sync()
        # host buffers, issued back to back, one synchronize at the end
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        S, psi, Gp = pin(c.S), pin(c.psi), pin(G)
        got, keep = [], []   # host inputs must live until the stream has passed the calls
        for t_lo, t_hi, ts in sets:
            nt, nq = t_hi - t_lo + 1, len(c.k)
            ins = torch.empty((nt, nq, 3, 192), dtype=torch.complex128).pin_memory()
            spec = torch.empty((nq, 3, 192), dtype=torch.complex128).pin_memory()
            comb = torch.empty((nt, 3, nq, nq), dtype=torch.complex128).pin_memory()
            ctx.insertion(S, psi, t_lo, t_hi, c.r, c.k, prec=prec, out=ins)
            eta = pin(c.eta(ts))
            keep.append(eta)
            ctx.spectator(S, eta, ts, c.r, c.k, prec=prec, out=spec)
            ctx.combine(spec, ins, Gp, Gp, Gp, prec=prec, out=comb)   # reads the two host outputs above
            got.append((ins, spec, comb))
        torch.cuda.synchronize()
        ctx.sync()
    for (ri, rs, rc), (gi, gs, gc) in zip(ref, got):
        assert torch.equal(ri, gi)
        assert torch.equal(rs, gs)
        assert torch.equal(rc, gc)
