"""Staged propagator slices (lhc_prop_stage): calls that read the complex64 copy give the
bits of the same calls that narrow the propagator themselves, including slice ranges that
wrap around T, calls that leave the staged range, a batch and a second context; staging
again follows a changed propagator; and the oracle agrees within the mixed tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_staged_slices_give_the_same_bits():
    from paper_1711_02384_gb300 import lhc
    c = CS.Case(6, 8, 3, lhc.momenta(8), seed=2600, r=(2, 0, 5, 0))
    S, psi, eta = dev(c.S), dev(c.psi), dev(c.eta(3))
    with lhc.Context(0) as ctx, lhc.Context(0) as other:
        for x in (ctx, other):
            x.set_projection("gemm")
        ref_i = ctx.insertion(S, psi, 1, 5, c.r, c.k, prec="mixed")
        ref_s = ctx.spectator(S, eta, 3, c.r, c.k, prec="mixed")
        ref_w = ctx.insertion(S, psi, 7, 8, c.r, c.k, prec="mixed")      # slices 7, 0
        ref_o = ctx.insertion(S, psi, 5, 7, c.r, c.k, prec="mixed")      # 7 lies outside 0..6
        ctx.stage_propagator(S, 0, 6)
        assert torch.equal(ctx.insertion(S, psi, 1, 5, c.r, c.k, prec="mixed"), ref_i)
        assert torch.equal(ctx.spectator(S, eta, 3, c.r, c.k, prec="mixed"), ref_s)
        assert torch.equal(ctx.insertion(S, psi, 5, 7, c.r, c.k, prec="mixed"), ref_o)
        assert torch.equal(other.insertion(S, psi, 1, 5, c.r, c.k, prec="mixed"), ref_i)   # another context
        got = ctx.batch([dict(part="ins", S=S, vec=psi, t_lo=1, t_hi=5, r=c.r, k=c.k),
                         dict(part="spec", S=S, vec=eta, t_lo=3, t_hi=3, r=c.r, k=c.k)])
        assert torch.equal(got[0], ref_i) and torch.equal(got[1], ref_s)
        ctx.stage_propagator(S, 6, 9)                                      # slices 6, 7, 0, 1
        assert torch.equal(ctx.insertion(S, psi, 7, 8, c.r, c.k, prec="mixed"), ref_w)
        # a changed propagator, staged again, is followed
        S.mul_(0.5)
        ctx.stage_propagator(S, 6, 9)
        half = ctx.insertion(S, psi, 7, 8, c.r, c.k, prec="mixed")
        ctx.unstage_propagator(S)
        assert torch.equal(half, ctx.insertion(S, psi, 7, 8, c.r, c.k, prec="mixed"))
        with pytest.raises(lhc.LhcError) as e:
            ctx.unstage_propagator(S)
        assert e.value.status == lhc.ENOTFOUND
        ctx.sync()
    assert CS.block_err(ref_i.cpu().numpy(), c.ref_insertion(1, 5), 2) < CS.MIXED_TOL
    assert CS.block_err(half.cpu().numpy() * 2, c.ref_insertion(7, 8), 2) < CS.MIXED_TOL


def test_stage_rejects_complex64_and_host_buffers():
    from paper_1711_02384_gb300 import lhc
    c = CS.Case(4, 4, 2, lhc.momenta(2), seed=2601)
    with lhc.Context(0) as ctx:
        with pytest.raises(lhc.LhcError):
            ctx.stage_propagator(dev(c.S.astype(np.complex64)), 0, 1)
        with pytest.raises(lhc.LhcError):
            ctx.stage_propagator(torch.from_numpy(c.S), 0, 1)
