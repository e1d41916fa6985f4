"""Long site ranges per CTA.  The fused kernel drains its tensor-memory accumulator into
an FP32 running sum that restarts after groups of at most 64 drained chunks; the group
sums add up in tensor memory when a chunk has at most 32 momentum representatives, and in
the CTA's block of partial sums in global memory (float4 atomic adds) for wider chunks.

With one site split per slice (LHC_NSPLIT=1) every CTA of a 24^3 slice runs all 864
k-steps: the meson spectator (drained every 2 k-steps) makes 432 chunks in 7 groups, the
insertion and the baryon spectator (every 4) 216 chunks in 4 groups.  Both second-level
paths must match the oracle within the mixed bound, as closely as the default launch
shape does, and repeat bit for bit (each partial-sum address has one writer, so the order
of the adds is fixed)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n2, path", [(4, "tensor memory: 17 representatives, chunk of 24"),
                                      (8, "global memory: 47 representatives, chunk of 48")])
def test_meson_parts_one_split_per_slice(monkeypatch, n2, path):
    from paper_1711_02384_gb300 import lhc
    c = CS.Case(24, 2, 2, lhc.momenta(n2), seed=3600 + n2, dtype=np.complex64, r=(3, 17, 8, 0))
    S, psi, eta = dev(c.S), dev(c.psi), dev(c.eta(1))
    with lhc.Context(0) as ctx:
        default = (ctx.insertion(S, psi, 0, 0, c.r, c.k), ctx.spectator(S, eta, 1, c.r, c.k))
        monkeypatch.setenv("LHC_NSPLIT", "1")
        runs = [(ctx.insertion(S, psi, 0, 0, c.r, c.k), ctx.spectator(S, eta, 1, c.r, c.k)) for _ in range(2)]
        ctx.sync()
    for a, b in zip(runs[0], runs[1]):
        assert torch.equal(a, b), "the same call differs between two runs"
    ri, rs = c.ref_insertion(0, 0), c.ref_spectator_meson(1)
    e_ins, e_spec = CS.block_err(runs[0][0].cpu().numpy(), ri, 2), CS.block_err(runs[0][1].cpu().numpy(), rs, 1)
    d_ins, d_spec = CS.block_err(default[0].cpu().numpy(), ri, 2), CS.block_err(default[1].cpu().numpy(), rs, 1)
    print(f"[parity] 24^3, one split per slice, {path}: insertion {e_ins:.3e} (default shape {d_ins:.3e}), "
          f"spectator {e_spec:.3e} (default shape {d_spec:.3e})")
    assert e_ins < CS.MIXED_TOL and e_spec < CS.MIXED_TOL
    # the long ranges sum as accurately as the short ones, within a margin
    assert e_ins < 1.5 * d_ins + 5e-8 and e_spec < 1.5 * d_spec + 5e-8


def test_baryon_spectator_one_split_per_slice(monkeypatch):
    """The baryon spectator with 123 momenta (62 representatives: two chunks of 32, the
    tensor-memory path) and 216 chunks per CTA."""
    from paper_1711_02384_gb300 import lhc
    c = CS.Case(24, 2, 2, lhc.momenta(9, 3), seed=3700, dtype=np.complex64, r=(5, 0, 19, 0))
    S, SB, eta = dev(c.S), dev(c.SB), dev(c.eta(0))
    with lhc.Context(0) as ctx:
        monkeypatch.setenv("LHC_NSPLIT", "1")
        runs = [ctx.spectator(S, eta, 0, c.r, c.k, GB=SB) for _ in range(2)]
        ctx.sync()
    assert torch.equal(runs[0], runs[1]), "the same call differs between two runs"
    e = CS.block_err(runs[0].cpu().numpy(), c.ref_spectator_baryon(0), 1)
    print(f"[parity] 24^3 baryon spectator, one split per slice: {e:.3e}")
    assert e < CS.MIXED_TOL
