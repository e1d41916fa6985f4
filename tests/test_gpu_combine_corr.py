"""Per-correlator parity of the combine (Eqs. 5 and 8) at the benchmark's shape: 93 sink
x 93 insertion momenta (|k|^2 <= 8), 16 noises, the 16 Dirac structures at sink and
source.  Every correlator C[t][g][p][q] is compared with the oracle's on its own,
relative to the largest |C| of its row (FP64 path 1e-12, mixed path 1e-6), for the
closed combine and both open-source-spin combines."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS
from oracle import contractions as OC
from paper_1711_02384_gb300 import inputs

pytestmark = pytest.mark.gpu

NQ, N_R = 93, 16


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def ctx():
    from paper_1711_02384_gb300 import lhc
    c = lhc.Context(0)
    yield c
    c.sync()
    c.close()


@pytest.fixture(scope="module")
def meson_parts():
    spec = inputs.gaussian_array(2400, 12, (NQ, N_R, 192))
    ins = inputs.gaussian_array(2401, 12, (2, NQ, N_R, 192))
    return spec, ins


@pytest.mark.parametrize("prec,tol", [("fp64", CS.FP64_TOL), ("mixed", CS.MIXED_TOL)])
def test_combine_headline_shape(ctx, meson_parts, prec, tol):
    spec, ins = meson_parts
    g16 = inputs.dirac_structures()
    g4 = np.broadcast_to(inputs.dirac_matrices()[3], (16, 4, 4)).copy()
    got = ctx.combine(dev(spec), dev(ins), dev(g16), dev(g4), dev(g16), prec=prec).cpu().numpy()
    ctx.sync()
    assert got.shape == (2, 16, NQ, NQ)
    worst = 0.0
    for t in range(2):
        ref = OC.combine_meson(spec, ins[t], g16, g4, g16)
        worst = max(worst, CS.corr_err(got[t], ref))
    print(f"[parity] combine 93x93x16, N_r=16, {prec}: worst per-correlator error {worst:.2e}")
    assert worst < tol


@pytest.mark.parametrize("prec,tol", [("fp64", CS.FP64_TOL), ("mixed", CS.MIXED_TOL)])
def test_open_combine_headline_shape(ctx, meson_parts, prec, tol):
    spec, ins = meson_parts
    g16 = inputs.dirac_structures()
    gs, gi = g16[[0, 5, 10, 15]], g16[[3, 6, 9, 12]]
    op = ctx.combine_open(dev(spec), dev(ins[:1]), dev(gs), dev(gi), prec=prec).cpu().numpy()[0]
    ctx.sync()
    worst = 0.0
    for a, c in ((0, 0), (1, 7), (2, 13), (3, 4)):
        for b in range(4):
            got = np.einsum("pqab,ba->pq", op[a, b], g16[c])
            ref = OC.combine_meson(spec, ins[0], gs[a:a + 1], gi[b:b + 1], g16[c:c + 1])[0]
            worst = max(worst, CS.corr_err(got, ref))
    print(f"[parity] open combine 93x93, N_r=16, {prec}: worst per-correlator error {worst:.2e}")
    assert worst < tol


@pytest.mark.parametrize("prec,tol", [("fp64", CS.FP64_TOL), ("mixed", CS.MIXED_TOL)])
def test_open_baryon_combine_headline_shape(ctx, meson_parts, prec, tol):
    _, ins = meson_parts
    spec = inputs.gaussian_array(2402, 12, (NQ, N_R, 3072))
    ws = inputs.gaussian_array(2403, 12, (2, 4, 4, 4))
    gi = inputs.dirac_structures()[[3, 8]]
    wc = inputs.gaussian_array(2404, 12, (2, 4, 4, 4))
    op = ctx.combine_open_baryon(dev(spec), dev(ins[:1]), dev(ws), dev(gi), prec=prec).cpu().numpy()[0]
    ctx.sync()
    worst = 0.0
    for a in range(2):
        for b in range(2):
            for w in wc:
                got = np.einsum("pqxyz,xyz->pq", op[a, b], w)
                ref = OC.combine_baryon(spec, ins[0], ws[a:a + 1], gi[b:b + 1], w[None])[0]
                worst = max(worst, CS.corr_err(got, ref))
    print(f"[parity] open baryon combine 93x93, N_r=16, {prec}: worst per-correlator error {worst:.2e}")
    assert worst < tol
