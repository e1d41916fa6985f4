"""Open-source-spin combine (the open-spin step of Eq. 8 extended to the source side):
contracting its output with any Gamma_src gives the combine of that structure, for every
pair of sink and insertion structures in the lists, against the library's combine and
the oracle's; and the full sweep over the 16 Dirac matrices."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS
from oracle import contractions as OC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1711_02384_gb300 import lhc
    c = lhc.Context(0)
    yield c
    c.sync()
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def parts():
    from oracle.momenta import momenta
    c = CS.Case(4, 8, 5, momenta(2), seed=2100, r=(1, 3, 0, 0))
    return c.ref_spectator_meson(5), c.ref_insertion(2, 5)      # [np][n_r][192], [nt][nq][n_r][192]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_open_combine_contracts_to_combine(ctx, parts, prec, tol):
    spec, ins = parts
    gs = CS.random_gammas(2101, 3, (4, 4))
    gi = CS.random_gammas(2102, 2, (4, 4))
    gc = CS.random_gammas(2103, 1, (4, 4))[0]
    op = ctx.combine_open(dev(spec), dev(ins), dev(gs), dev(gi), prec=prec).cpu().numpy()
    ctx.sync()
    assert op.shape == (4, 3, 2, spec.shape[0], ins.shape[1], 4, 4)
    for a in range(3):
        for b in range(2):
            got = np.einsum("tpqab,ba->tpq", op[:, a, b], gc)
            ref = np.stack([OC.combine_meson(spec, ins[t], gs[a:a + 1], gi[b:b + 1], gc[None])[0]
                            for t in range(ins.shape[0])])
            assert CS.corr_err(got, ref) < tol
            lib = ctx.combine(dev(spec), dev(ins), dev(gs[a:a + 1]), dev(gi[b:b + 1]), dev(gc[None]),
                              prec=prec).cpu().numpy()[:, 0]
            assert CS.corr_err(got, lib) < (1e-12 if prec == "fp64" else 2 * tol)


def test_dirac_basis_sweep(ctx, parts):
    """All 16 x 16 x 16 (Gamma_snk, Gamma_ins, Gamma_src) products of the Dirac basis from
    one open call, spot-checked against the oracle's combine."""
    spec, ins = parts
    g16 = CS.gamma16()
    op = ctx.combine_open(dev(spec), dev(ins[:1]), dev(g16), dev(g16), prec="fp64").cpu().numpy()[0]
    ctx.sync()
    C = np.einsum("sipqab,cba->sicpq", op, g16)                  # [snk][ins][src][p][q]
    rng = np.random.default_rng(2104)
    for s, i, c in rng.integers(0, 16, size=(12, 3)):
        ref = OC.combine_meson(spec, ins[0], g16[s:s + 1], g16[i:i + 1], g16[c:c + 1])[0]
        assert CS.corr_err(C[s, i, c], ref) < CS.FP64_TOL


@pytest.fixture(scope="module")
def baryon_parts():
    from oracle.momenta import momenta
    c = CS.Case(4, 8, 5, momenta(2), seed=2110, r=(2, 0, 1, 0))
    return c.ref_spectator_baryon(5), c.ref_insertion(2, 5)     # [np][n_r][3072], [nt][nq][n_r][192]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_open_baryon_combine_contracts_to_combine(ctx, baryon_parts, prec, tol):
    """Contracting the open (a1, a2, b) source spins with any W_src gives the baryon combine
    of Eq. 8 for that structure: against the oracle and the library's closed combine."""
    spec, ins = baryon_parts
    ws = CS.random_gammas(2111, 2, (4, 4, 4))
    gi = CS.random_gammas(2112, 3, (4, 4))
    wc = CS.random_gammas(2113, 2, (4, 4, 4))
    op = ctx.combine_open_baryon(dev(spec), dev(ins), dev(ws), dev(gi), prec=prec).cpu().numpy()
    ctx.sync()
    assert op.shape == (4, 2, 3, spec.shape[0], ins.shape[1], 4, 4, 4)
    for a in range(2):
        for b in range(3):
            for w in wc:
                got = np.einsum("tpqxyz,xyz->tpq", op[:, a, b], w)
                ref = np.stack([OC.combine_baryon(spec, ins[t], ws[a:a + 1], gi[b:b + 1], w[None])[0]
                                for t in range(ins.shape[0])])
                assert CS.corr_err(got, ref) < tol
                lib = ctx.combine(dev(spec), dev(ins), dev(ws[a:a + 1]), dev(gi[b:b + 1]), dev(w[None]),
                                  prec=prec).cpu().numpy()[:, 0]
                assert CS.corr_err(got, lib) < (1e-12 if prec == "fp64" else 2 * tol)


def test_open_baryon_single_slice_and_ragged(ctx, baryon_parts):
    """One insertion slice (no nt axis), one noise, and momentum lists that leave ragged
    row and column tiles (16 np and 4 nq not multiples of the 32 x 48 tile)."""
    spec, ins = baryon_parts
    spec1, ins1 = spec[:3, :1], ins[1, :5, :1]
    ws = CS.random_gammas(2114, 1, (4, 4, 4))
    gi = CS.random_gammas(2115, 1, (4, 4))
    op = ctx.combine_open_baryon(dev(spec1), dev(ins1), dev(ws), dev(gi), prec="fp64").cpu().numpy()
    ctx.sync()
    assert op.shape == (1, 1, 3, 5, 4, 4, 4)
    # W[a1'][a2'][b'] = xyz, Gamma_ins = uv, B[p][a1',a1,a2',a2,b',c] = pxjyhzc, I[q][u,v,b,c]
    ref = np.einsum("xyz,uv,pxjyhzc,quvbc->pqjhb", ws[0], gi[0],
                    spec1[:, 0].reshape(3, 4, 4, 4, 4, 4, 3), ins1[:, 0].reshape(5, 4, 4, 4, 3))
    assert CS.corr_err(np.moveaxis(op[0, 0], 1, -1), np.moveaxis(ref, 1, -1)) < CS.FP64_TOL
