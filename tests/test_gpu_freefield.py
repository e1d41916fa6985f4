"""End to end on the GPU with real free-field solves: the library's Wilson-Dirac
operator and solver (unit links) produce the point-to-all propagator and the solutions of
fully diluted noise; the library's spectator, insertion and combine then reproduce the
free three-point function evaluated independently in momentum space (convolution
theorem).  Operator and propagator are also checked against the oracle's stencil and
closed form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _pins as P
from oracle import freefield as F
from oracle import gamma as OG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1711_02384_gb300 import lhc
    c = lhc.Context(0)
    yield c
    c.sync()
    c.close()


def _gammas(basis):
    if basis == "rotated":
        # U gamma U^dagger for a random unitary U: a valid Hermitian basis whose matrices
        # are dense (the library's general stencil; the other two take its sparse one)
        rng = np.random.default_rng(7)
        q, _ = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
        return np.array([q @ g @ q.conj().T for g in OG.chiral()])
    return np.array(OG.chiral() if basis == "chiral" else OG.dirac_pauli())


@pytest.mark.parametrize("basis", ["chiral", "dirac_pauli", "rotated"])
@pytest.mark.parametrize("dagger", [False, True])
def test_wilson_operator_matches_stencil(ctx, basis, dagger):
    L, T, m = 4, 6, 0.3
    g = _gammas(basis)
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((2, T, L ** 3, 12)) + 1j * rng.standard_normal((2, T, L ** 3, 12))
    got = ctx.wilson_apply(torch.from_numpy(psi).cuda(), m, g, dagger=dagger).cpu().numpy()
    ctx.sync()
    gs = [-x for x in g] if dagger else list(g)    # D^dagger: gamma_mu -> -gamma_mu
    for n in range(2):
        f = psi[n].reshape(T, L, L, L, 4, 3)
        ref = F.apply_wilson(f, m, gs).reshape(T, L ** 3, 12)
        assert np.max(np.abs(got[n] - ref)) < 1e-13 * np.max(np.abs(ref))


def test_point_to_all_propagator_matches_closed_form(ctx):
    L, T, m = 4, 8, 0.3
    g = _gammas("chiral")
    V3 = L ** 3
    r, r4 = (1, 2, 3), 1
    rsite = (r[2] * L + r[1]) * L + r[0]
    src = np.zeros((12, T, V3, 12), dtype=complex)
    for sc in range(12):
        src[sc, r4, rsite, sc] = 1.0
    sol, it, res = ctx.wilson_solve(torch.from_numpy(src).cuda(), m, g, tol=1e-13)
    ctx.sync()
    assert res < 1e-11, (it, res)
    G = np.transpose(sol.cpu().numpy(), (1, 2, 3, 0))          # [T][V3][sink 12][source 12]
    ff = P.FreeField(L=L, T=T, m=m)
    sites = np.arange(V3)
    for t in range(T):
        ref = ff.G(t, sites, r4, np.full(V3, rsite), rotate=False)
        assert np.max(np.abs(G[t] - ref)) < 1e-10, t


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_factorized_free_correlator_end_to_end(ctx, prec, tol):
    """Everything on the GPU: propagator and solutions from the library's solver (full
    spin-colour-site dilution on the sink slice, 768 noises), then spectator, insertion
    and combine; against the momentum-space free correlator."""
    L, T, m = 4, 8, 0.3
    g = _gammas("chiral")
    V3, N = L ** 3, 12 * L ** 3
    r, r4, tf, ty = (1, 2, 3), 1, 5, 3
    rsite = (r[2] * L + r[1]) * L + r[0]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    src = np.zeros((12, T, V3, 12), dtype=complex)
    for sc in range(12):
        src[sc, r4, rsite, sc] = 1.0
    sol, _, res = ctx.wilson_solve(dev(src), m, g, tol=1e-13)
    assert res < 1e-11
    S = sol.permute(1, 2, 3, 0).contiguous()                   # G(x, r): [T][V3][12][12]
    eta = np.zeros((N, V3, 12), dtype=complex)                 # unit noise on every (site, spin, colour)
    for x0 in range(V3):
        for sc in range(12):
            eta[x0 * 12 + sc, x0, sc] = 1.0
    src_t = torch.zeros((N, T, V3, 12), dtype=torch.complex128, device="cuda")
    src_t[:, tf] = dev(eta)
    psi, _, res = ctx.wilson_solve(src_t, m, g, tol=1e-13)
    assert res < 1e-11
    k = np.asarray(P.M.momenta(2)[:7], dtype=np.int32)
    r4v = np.array([r[0], r[1], r[2], r4], dtype=np.int32)
    spec = ctx.spectator(S, dev(eta), tf, r4v, k, prec=prec)
    ins = ctx.insertion(S, psi, ty, ty, r4v, k, prec=prec)
    rng = np.random.default_rng(6)
    gs, gi, gc = (rng.standard_normal((1, 4, 4)) + 1j * rng.standard_normal((1, 4, 4)) for _ in range(3))
    c = ctx.combine(spec, ins, dev(gs), dev(gi), dev(gc), prec=prec)
    got = N * c.cpu().numpy()[0, 0]
    ctx.sync()
    ref = P.FreeField(L=L, T=T, m=m).momentum_space_3pt(r4, r, tf, ty, gs[0], gi[0], gc[0], k, k)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"free correlator end to end ({prec}): relative error {err:.3e}")
    assert err < tol


def test_forward_and_backward_in_one_pass(ctx):
    """Noise on two sink slices at once (x4' before the source, x4'' after it, as in the
    paper's runs): one set of solves, one insertion call over x4' .. x4'' and one spectator
    call per sink slice give both the backward and the forward three-point functions,
    each equal to its momentum-space free correlator (full dilution on both slices, 1536
    noises; the noises of one slice contribute nothing to the other's spectator)."""
    L, T, m = 4, 8, 0.3
    g = _gammas("chiral")
    V3 = L ** 3
    r, r4, tb, tfw = (2, 1, 3), 3, 1, 5          # backward sink 1, source 3, forward sink 5
    rsite = (r[2] * L + r[1]) * L + r[0]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    src = np.zeros((12, T, V3, 12), dtype=complex)
    for sc in range(12):
        src[sc, r4, rsite, sc] = 1.0
    sol, _, res = ctx.wilson_solve(dev(src), m, g, tol=1e-13)
    assert res < 1e-11
    S = sol.permute(1, 2, 3, 0).contiguous()
    N1 = 12 * V3
    eta = torch.zeros((2 * N1, T, V3, 12), dtype=torch.complex128, device="cuda")
    unit = torch.zeros((N1, V3, 12), dtype=torch.complex128)
    for x0 in range(V3):
        for sc in range(12):
            unit[x0 * 12 + sc, x0, sc] = 1.0
    eta[:N1, tb] = unit.cuda()
    eta[N1:, tfw] = unit.cuda()
    psi, _, res = ctx.wilson_solve(eta, m, g, tol=1e-13)
    assert res < 1e-11
    k = np.asarray(P.M.momenta(1), dtype=np.int32)
    r4v = np.array([r[0], r[1], r[2], r4], dtype=np.int32)
    ins = ctx.insertion(S, psi, tb, tfw, r4v, k, prec="fp64")                 # slices 1 .. 5, one call
    rng = np.random.default_rng(7)
    gs, gi, gc = (rng.standard_normal((1, 4, 4)) + 1j * rng.standard_normal((1, 4, 4)) for _ in range(3))
    ff = P.FreeField(L=L, T=T, m=m)
    for tsink, ty in ((tb, 2), (tfw, 4)):
        spec = ctx.spectator(S, eta[:, tsink].contiguous(), tsink, r4v, k, prec="fp64")
        c = ctx.combine(spec, ins[ty - tb], dev(gs), dev(gi), dev(gc), prec="fp64")
        got = 2 * N1 * c.cpu().numpy()[0]
        ref = ff.momentum_space_3pt(r4, r, tsink, ty, gs[0], gi[0], gc[0], k, k)
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref), (tsink, ty)
    ctx.sync()
