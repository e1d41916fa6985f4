"""Batched calls (lhc_batch): many mixed-precision insertion and spectator calls with
uneven momentum sets, lattices and parts in one persistent fused launch per part kind and
momentum-chunk width;
the results must equal, bit for bit, those of the same calls made one by one with the
tensor-core projection, also when replayed from a CUDA graph, and the oracle within the
mixed tolerance."""
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


def test_persistent_batch_replayed_from_a_cuda_graph():
    """Persistent launches (one per part kind and chunk width) over calls with five
    momentum-chunk widths (7, 33, 57, 93 and 147 momenta: 4, 17, 29, 47 and 74
    representatives, chunks of 8, 24, 32, 48 and two of 40), two lattices and both input
    precisions, captured in a CUDA graph and replayed:
    the replay equals the same calls made one by one bit for bit, and the oracle within
    the mixed tolerance."""
    from paper_1711_02384_gb300 import lhc
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sets = [lhc.momenta(1), lhc.momenta(3), lhc.momenta(5), lhc.momenta(8), lhc.momenta(10)]
    cases = [CS.Case(6, 6, 3, sets[0], seed=2510, r=(1, 0, 5, 0)),
             CS.Case(8, 4, 2, sets[3], seed=2511, r=(3, 2, 1, 0), dtype=np.complex64)]
    calls = []
    for n, c in enumerate(cases):
        S, SB, psi, eta = dev(c.S), dev(c.SB), dev(c.psi), dev(c.eta(1))
        for m, k in enumerate(sets):
            t_lo = (n + m) % c.T
            calls.append(dict(part="ins", S=S, vec=psi, t_lo=t_lo, t_hi=t_lo + 1 + m % 2, r=c.r, k=k))
            calls.append(dict(part="spec", S=S, vec=eta, t_lo=1, t_hi=1, r=c.r, k=k))
        calls.append(dict(part="baryon", S=S, GB=SB, vec=eta, t_lo=1, t_hi=1, r=c.r, k=sets[2 + n]))
    stream = torch.cuda.Stream()
    with lhc.Context(0) as ctx, torch.cuda.stream(stream):
        ctx.set_projection("gemm")
        ref = []
        for c in calls:
            if c["part"] == "ins":
                ref.append(ctx.insertion(c["S"], c["vec"], c["t_lo"], c["t_hi"], c["r"], c["k"], prec="mixed",
                                         stream=stream.cuda_stream))
            else:
                ref.append(ctx.spectator(c["S"], c["vec"], c["t_lo"], c["r"], c["k"], prec="mixed", GB=c.get("GB"),
                                         stream=stream.cuda_stream))
        outs = ctx.batch(calls, stream=stream.cuda_stream)   # phase tables and workspace for the capture
        for c, o in zip(calls, outs):
            c["out"] = o
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            ctx.batch(calls, stream=stream.cuda_stream)
        for o in outs:
            o.fill_(float("nan"))
        graph.replay()
        stream.synchronize()
        ctx.sync(stream.cuda_stream)
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
        graph.replay()                                          # a second replay, the same bits
        stream.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
    # calls 17 and 21: the 93-momentum insertion over slices 0..2 and the baryon of the
    # second lattice; call 1: the 7-momentum meson spectator of the first
    c = cases[1]
    assert CS.block_err(outs[17].cpu().numpy(), c.ref_insertion(0, 2), 2) < CS.MIXED_TOL
    assert CS.block_err(outs[21].cpu().numpy(), c.ref_spectator_baryon(1), 1) < CS.MIXED_TOL
    c = cases[0]
    assert CS.block_err(outs[1].cpu().numpy(), c.ref_spectator_meson(1), 1) < CS.MIXED_TOL


def test_batch_with_a_call_that_fills_the_gpu():
    """A call whose own launch fills several waves of the GPU (16^3, 32 noises, 8 slices)
    keeps its own fused launch inside the batch; the small calls beside it share a
    persistent launch.  Every output equals the same call made alone, bit for bit."""
    from paper_1711_02384_gb300 import lhc, inputs
    dev = torch.device("cuda", 0)
    L, T, NR = 16, 8, 32
    V3 = L ** 3
    S = torch.from_numpy(inputs.propagator(2520, L, T).astype(np.complex64)).to(dev)
    psi = torch.from_numpy(inputs.solutions(2521, L, T, NR).astype(np.complex64)).to(dev)
    eta = torch.from_numpy(inputs.noise(2522, L, 4, 3).astype(np.complex64)).to(dev)
    k93, k7 = lhc.momenta(8), lhc.momenta(1)
    calls = [dict(part="ins", S=S, vec=psi, t_lo=0, t_hi=7, r=(1, 2, 3, 0), k=k93),
             dict(part="spec", S=S, vec=eta, t_lo=3, t_hi=3, r=(1, 2, 3, 0), k=k7),
             dict(part="spec", S=S, vec=eta, t_lo=3, t_hi=3, r=(0, 5, 1, 0), k=k93)]
    with lhc.Context(0) as ctx:
        ctx.set_projection("gemm")
        got = ctx.batch(calls)
        ref = [ctx.insertion(S, psi, 0, 7, calls[0]["r"], k93, prec="mixed"),
               ctx.spectator(S, eta, 3, calls[1]["r"], k7, prec="mixed"),
               ctx.spectator(S, eta, 3, calls[2]["r"], k93, prec="mixed")]
        ctx.sync()
    assert got[0].shape == (8, len(k93), NR, 192)
    for g, r in zip(got, ref):
        assert torch.equal(g, r)
