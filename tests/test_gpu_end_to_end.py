"""End to end on the benchmark's lattice (24^3, 16 noises, 93 momenta, complex128): the
mixed insertion of one slice and the meson spectator of the sink slice computed on the
GPU, then combined there for the 16 Dirac structures at sink and source with gamma_4 at
the insertion (Eqs. 10, 9 and 5), against the oracle's whole chain on the same inputs.
Every correlator C[g][p][q] must be within 1e-6 of the oracle's, relative to the largest
|C| of its row; the parts within 1e-6 per (momentum) block.  The errors of both parts
add up in the combine, so this is the check that binds the mixed path's drain interval."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def block_err(got, want):
    got, want = got.reshape(want.shape[0], -1), want.reshape(want.shape[0], -1)
    return float(np.max(np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)))


@pytest.mark.parametrize("seed", [2900, 2950, 3000])
def test_chain_24c_one_slice_per_correlator(seed):
    from oracle import contractions as OC
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import inputs, lhc
    L, n_r, t_ins, t_snk = 24, 16, 5, 10
    k = momenta(8)
    S = inputs.propagator(seed, L, 48, slices=[t_ins, t_snk])          # as a 2-slice lattice
    psi = inputs.solutions(seed + 1, L, 48, n_r, slices=[t_ins, t_snk])   # [n_r][T = 2][V3][12]
    eta = inputs.noise(seed + 2, L, n_r, t_snk)
    g16 = inputs.dirac_structures()
    g4 = np.broadcast_to(inputs.dirac_matrices()[3], (16, 4, 4)).copy()
    r = np.zeros(4, dtype=np.int32)
    with lhc.Context(0) as ctx:
        dS = dev(S)
        gi = ctx.insertion(dS, dev(psi), 0, 0, r, k, prec="mixed")
        gs = ctx.spectator(dS, dev(eta), 1, r, k, prec="mixed")
        gc = ctx.combine(gs, gi, dev(g16), dev(g4), dev(g16), prec="mixed")
        gi, gs, gc = gi.cpu().numpy(), gs.cpu().numpy(), gc.cpu().numpy()
        ctx.sync()
    g5 = CS.g5_matrix()
    ri = OC.insertion(S[0:1], psi[:, 0:1], g5, r[:3], k, L)
    rs = OC.spectator_meson(S[1], eta, g5, r[:3], k, L)
    rc = OC.combine_meson(rs, ri[0], g16, g4, g16)
    e_ins, e_spec, e_corr = block_err(gi[0], ri[0]), block_err(gs, rs), CS.corr_err(gc[0], rc)
    print(f"[parity] 24^3 chain, seed {seed}: insertion {e_ins:.3e}, spectator {e_spec:.3e}, "
          f"combine {e_corr:.3e} per correlator")
    assert e_ins < CS.MIXED_TOL and e_spec < CS.MIXED_TOL
    assert e_corr < CS.MIXED_TOL


def test_chain_48c_largest_served_lattice_per_correlator():
    """The meson chain on the largest served lattice (48^3, 110592 sites per slice: the
    longest site sums), 4 noises, complex64 inputs, 93 momenta, against the oracle on the
    same complex64-rounded inputs, per correlator."""
    from oracle import contractions as OC
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import inputs, lhc
    L, n_r = 48, 4
    k = momenta(8)
    S = inputs.propagator(3100, L, 96, slices=[20, 30]).astype(np.complex64)
    psi = inputs.solutions(3101, L, 96, n_r, slices=[20, 30]).astype(np.complex64)
    eta = inputs.noise(3102, L, n_r, 30).astype(np.complex64)
    g16 = inputs.dirac_structures()
    g4 = np.broadcast_to(inputs.dirac_matrices()[3], (16, 4, 4)).copy()
    r = np.array([7, 30, 41, 0], dtype=np.int32)
    with lhc.Context(0) as ctx:
        dS = dev(S)
        gi = ctx.insertion(dS, dev(psi), 0, 0, r, k, prec="mixed")
        gs = ctx.spectator(dS, dev(eta), 1, r, k, prec="mixed")
        gc = ctx.combine(gs, gi, dev(g16), dev(g4), dev(g16), prec="mixed")
        gi, gs, gc = gi.cpu().numpy(), gs.cpu().numpy(), gc.cpu().numpy()
        ctx.sync()
    g5 = CS.g5_matrix()
    ri = OC.insertion(S[0:1].astype(complex), psi[:, 0:1].astype(complex), g5, r[:3], k, L)
    rs = OC.spectator_meson(S[1].astype(complex), eta.astype(complex), g5, r[:3], k, L)
    rc = OC.combine_meson(rs, ri[0], g16, g4, g16)
    e_ins, e_spec, e_corr = block_err(gi[0], ri[0]), block_err(gs, rs), CS.corr_err(gc[0], rc)
    print(f"[parity] 48^3 chain: insertion {e_ins:.3e}, spectator {e_spec:.3e}, combine {e_corr:.3e} per correlator")
    assert e_ins < CS.MIXED_TOL and e_spec < CS.MIXED_TOL
    assert e_corr < CS.MIXED_TOL


@pytest.mark.parametrize("seed", [3300, 3400])
def test_baryon_chain_16c_123_momenta_per_correlator(seed):
    """The baryon chain on 16^3 with the 123 momenta of the baryon configuration (|k|^2 <= 9,
    |k_j| <= 3: 62 representatives, two chunks), 4 noises, complex64 propagators: the mixed
    eps-eps spectator and the insertion of one slice on the GPU, combined there for 4
    random sink/source structures and insertion Gammas, against the oracle's chain
    (Sec. 2, Eqs. 5, 8, 10), per correlator within 1e-6."""
    from oracle import contractions as OC
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import inputs, lhc
    L, n_r, t_ins, t_snk = 16, 4, 3, 9
    k = momenta(9, 3)
    GA = inputs.propagator(seed, L, 32, slices=[t_ins, t_snk]).astype(np.complex64)
    GB = inputs.propagator(seed, L, 32, slices=[t_ins, t_snk], tensor_id=inputs.TID_PROP_B).astype(np.complex64)
    psi = inputs.solutions(seed + 1, L, 32, n_r, slices=[t_ins, t_snk]).astype(np.complex64)
    eta = inputs.noise(seed + 2, L, n_r, t_snk).astype(np.complex64)
    ws = CS.random_gammas(seed + 3, 4, (4, 4, 4))
    gi = CS.random_gammas(seed + 4, 4, (4, 4))
    wc = CS.random_gammas(seed + 5, 4, (4, 4, 4))
    r = np.array([2, 5, 11, 0], dtype=np.int32)
    with lhc.Context(0) as ctx:
        dA = dev(GA)
        ins = ctx.insertion(dA, dev(psi), 0, 0, r, k, prec="mixed")
        spec = ctx.spectator(dA, dev(eta), 1, r, k, prec="mixed", GB=dev(GB))
        corr = ctx.combine(spec, ins, dev(ws), dev(gi), dev(wc), prec="mixed")
        # the source spins left open, W_src applied afterwards (on the host: a 64-term sum)
        op = ctx.combine_open_baryon(spec, ins, dev(ws), dev(gi), prec="mixed")[0]
        ins, spec, corr, op = ins.cpu().numpy(), spec.cpu().numpy(), corr.cpu().numpy(), op.cpu().numpy()
        ctx.sync()
    g5 = CS.g5_matrix()
    ri = OC.insertion(GA[0:1].astype(complex), psi[:, 0:1].astype(complex), g5, r[:3], k, L)
    rs = OC.spectator_baryon(GA[1].astype(complex), GB[1].astype(complex), eta.astype(complex), g5, r[:3], k, L)
    rc = OC.combine_baryon(rs, ri[0], ws, gi, wc)
    e_ins, e_spec, e_corr = block_err(ins[0], ri[0]), block_err(spec, rs), CS.corr_err(corr[0], rc)
    e_open = max(CS.corr_err(np.einsum("pqxyz,xyz->pq", op[g, g], wc[g]), rc[g]) for g in range(len(wc)))
    print(f"[parity] baryon 16^3 chain, 123 momenta, seed {seed}: insertion {e_ins:.3e}, spectator {e_spec:.3e}, "
          f"combine {e_corr:.3e}, open combine {e_open:.3e} per correlator")
    assert e_ins < CS.MIXED_TOL and e_spec < CS.MIXED_TOL
    assert e_corr < CS.MIXED_TOL and e_open < CS.MIXED_TOL
